// wf_device.cuh -- device building blocks of the GB300 messenger Wiener filter:
// complex arithmetic, register DFTs, a shared-memory Stockham FFT engine,
// the real<->complex row-transform wrappers and the device-resident state.
//
// The transforms are the flat-sky stand-ins for the spherical-harmonic
// transforms of Sec. 2 of Huffenberger 2017 (two transforms per iteration):
// a row-wise real DFT along x (the basis where horizontal stripes are
// diagonal) and a column DFT along y (completing the 2D DFT where the signal
// and the 1/f noise are diagonal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace wf {

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward transforms) or +i (inverse transforms)
template <bool INV>
__device__ __forceinline__ float2 rot90(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
template <bool INV>
__device__ __forceinline__ float2 tw_dir(float2 w) { return INV ? cconj(w) : w; }

// ---------------------------------------------------------------- small DFTs
// Forward DFTs use exp(-2 pi i nk/R); INV uses exp(+2 pi i nk/R); no scaling.
template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  float2 s13 = cadd(a1, a3), d13 = rot90<INV>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

// 3-point DFT: with w = exp(-+ 2 pi i / 3) = -1/2 -+ i sqrt(3)/2,
// X0 = a + b + c, X1 = a + w b + w^2 c, X2 = a + w^2 b + w c, i.e.
// X1,2 = a - (b + c)/2 -+ i (sqrt(3)/2)(b - c)  (forward: upper sign).
#define WF_S3 0.86602540378443865f
template <bool INV>
__device__ __forceinline__ void dft3(float2& a, float2& b, float2& c) {
  const float2 s = cadd(b, c), d = csub(b, c);
  const float2 m = make_float2(fmaf(-0.5f, s.x, a.x), fmaf(-0.5f, s.y, a.y));
  // -i (sqrt3/2) d (forward) or +i (sqrt3/2) d (inverse)
  const float2 r = INV ? make_float2(-WF_S3 * d.y, WF_S3 * d.x) : make_float2(WF_S3 * d.y, -WF_S3 * d.x);
  a = cadd(a, s);
  b = cadd(m, r);
  c = csub(m, r);
}

// cos(pi/4), cos(pi/8), sin(pi/8)
#define WF_C4 0.70710678118654752f
#define WF_C8 0.92387953251128674f
#define WF_S8 0.38268343236508977f

// multiply by W8^1 = exp(-+ i pi/4)
template <bool INV>
__device__ __forceinline__ float2 mul_w8_1(float2 a) {
  return INV ? make_float2(WF_C4 * (a.x - a.y), WF_C4 * (a.x + a.y))
             : make_float2(WF_C4 * (a.x + a.y), WF_C4 * (a.y - a.x));
}
// multiply by W8^3 = exp(-+ 3 i pi/4)
template <bool INV>
__device__ __forceinline__ float2 mul_w8_3(float2 a) {
  return INV ? make_float2(-WF_C4 * (a.x + a.y), WF_C4 * (a.x - a.y))
             : make_float2(WF_C4 * (a.y - a.x), -WF_C4 * (a.x + a.y));
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* a) {
  // even / odd halves, then combine with W8^k
  float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  float2 o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  o1 = mul_w8_1<INV>(o1);
  o2 = rot90<INV>(o2);
  o3 = mul_w8_3<INV>(o3);
  a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
  a[1] = cadd(e1, o1); a[5] = csub(e1, o1);
  a[2] = cadd(e2, o2); a[6] = csub(e2, o2);
  a[3] = cadd(e3, o3); a[7] = csub(e3, o3);
}

template <bool INV>
__device__ __forceinline__ float2 w16(int m, float2 a) {
  // multiply a by W16^m for the m that occur in the 4x4 split
  float2 w;
  switch (m) {
    case 1: w = make_float2(WF_C8, -WF_S8); break;
    case 2: w = make_float2(WF_C4, -WF_C4); break;
    case 3: w = make_float2(WF_S8, -WF_C8); break;
    case 4: w = make_float2(0.f, -1.f); break;
    case 6: w = make_float2(-WF_C4, -WF_C4); break;
    case 9: w = make_float2(-WF_C8, WF_S8); break;
    default: return a;
  }
  return cmul(a, tw_dir<INV>(w));
}

template <bool INV>
__device__ __forceinline__ void dft16(float2* a) {
  // 16 = 4 x 4: X[k1 + 4 k2] = sum_n2 W4^{n2 k2} W16^{n2 k1} sum_n1 a[4 n1 + n2] W4^{n1 k1}
  float2 y[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    float2 b0 = a[n2], b1 = a[n2 + 4], b2 = a[n2 + 8], b3 = a[n2 + 12];
    dft4<INV>(b0, b1, b2, b3);
    y[n2 * 4 + 0] = b0;
    y[n2 * 4 + 1] = w16<INV>(n2 * 1, b1);
    y[n2 * 4 + 2] = w16<INV>(n2 * 2, b2);
    y[n2 * 4 + 3] = w16<INV>(n2 * 3, b3);
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 c0 = y[0 * 4 + k1], c1 = y[1 * 4 + k1], c2 = y[2 * 4 + k1], c3 = y[3 * 4 + k1];
    dft4<INV>(c0, c1, c2, c3);
    a[k1] = c0; a[k1 + 4] = c1; a[k1 + 8] = c2; a[k1 + 12] = c3;
  }
}

template <int R, bool INV>
__device__ __forceinline__ void dftR(float2* u) {
  if constexpr (R == 3) dft3<INV>(u[0], u[1], u[2]);
  else if constexpr (R == 2) dft2<INV>(u[0], u[1]);
  else if constexpr (R == 4) dft4<INV>(u[0], u[1], u[2], u[3]);
  else if constexpr (R == 8) dft8<INV>(u);
  else if constexpr (R == 16) dft16<INV>(u);
}

// ---------------------------------------------------------------- FFT engine
// Shared-memory index padding: one extra slot every 16 complex values, so the
// strided scatters of the early Stockham stages do not pile onto one bank.
__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }
template <int L>
struct SPad { static constexpr int size = L + L / 16; };

// Radix of the stage that starts with sub-transform length NS.  Lengths are
// 2^k or 3 * 2^k: a factor 3 is taken by the first stage (E then holds a
// factor 3 too), the rest by powers of two up to the largest one dividing E.
template <int L, int E, int NS>
struct StageRadix {
  static_assert(L % 3 != 0 || E % 3 == 0, "lengths 3*2^k need a factor 3 in E");
  static constexpr int P2 = E & -E;  // largest power of two dividing E
  static constexpr int rem = L / NS;
  static constexpr int value = (NS == 1 && L % 3 == 0) ? 3 : (rem >= P2 ? P2 : rem);
};

// (L - k) mod L for 0 <= k < L: the index of the mode -k.
template <int L>
__device__ __forceinline__ int neg_mod(int k) { return k == 0 ? 0 : L - k; }

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialisation may start while the previous kernel on the stream is still
// running; pdl_wait() blocks until that kernel has completed and its writes
// are visible (a no-op for an ordinary launch), so everything before it may
// only touch shared memory and tables that no kernel of the iteration
// writes.  pdl_trigger() lets the next kernel start its own prologue.
// Every kernel launched this way calls pdl_wait() on every path, so the
// completion of the last kernel implies that of all before it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Twiddle read: read-only global path, or a plain load when the table has
// been staged in shared memory (TWS = true).
template <bool TWS>
__device__ __forceinline__ float2 tw_load(const float2* __restrict__ tab, int i) {
  if constexpr (TWS) return tab[i];
  else return __ldg(&tab[i]);
}

// Barrier between the exchange steps of a transform: the whole block, or
// only the warp when one warp owns the transform (WARP = true).
template <bool WARP>
__device__ __forceinline__ void fft_sync() {
  if constexpr (WARP) __syncwarp();
  else __syncthreads();
}

// 32-bit shared-memory address of a generic pointer into shared memory
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------- tensor-core radix-16
// A radix-16 stage as a matrix product on the tensor cores (DFT as GEMM): for
// the 32 length-16 DFTs held by one warp (one per lane, B = E/R = 1),
// Y[k][n] = sum_r W16^{kr} U[r][n], with complex values split into real
// products Yr = Fr Ur - Fi Ui, Yi = Fr Ui + Fi Ur, each an m16n8k8 TF32 MMA
// per 8 lanes (n) and 8 inputs (r), FP32 accumulation.  PREC = 1 splits both
// factors as x = hi + lo with hi = TF32(x), lo = TF32(x - hi) and sums
// hi*hi + hi*lo + lo*hi (about FP32 accuracy); PREC = 2 takes hi*hi alone
// (TF32 accuracy, 2^-11 relative per product).
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
template <int PREC>
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  if constexpr (PREC == 1) lo = to_tf32(x - __uint_as_float(hi));
  else lo = 0u;
}
// d += a b for one m16n8k8 tile: a 16 x 8 (row), b 8 x 8 (column), d 16 x 8.
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// d += a b with the split factors (PREC = 1: three products, small ones first)
template <int PREC>
__device__ __forceinline__ void mma_split(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                          uint32_t bh0, uint32_t bh1, uint32_t bl0, uint32_t bl1) {
  if constexpr (PREC == 1) {
    mma_tf32(d, al, bh0, bh1);
    mma_tf32(d, ah, bl0, bl1);
  }
  mma_tf32(d, ah, bh0, bh1);
}
__device__ __forceinline__ float2 lds_f2(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0,%1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void sts_f2(uint32_t addr, float2 v) {
  asm volatile("st.shared.v2.f32 [%0], {%1,%2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// The stage with sub-transform length NS of a length-L transform whose
// threads hold E = 16 values each.  Each lane's own inputs (twiddled as in the
// FP32 stage) are staged at 16 t + r of its transform's buffer; the lanes read
// the operand fragments of the warp's 32 transforms from there (addresses and
// t of the other lanes by shuffles, so any lane-to-transform layout works);
// after a block barrier the outputs go to their autosort positions.  Every
// thread of the block calls it; sb is free on entry.
template <int L, int NS, bool INV, bool TWS, int PREC>
__device__ __forceinline__ void tc_radix16_stage(float2 (&v)[16], float2* sb, int t,
                                                 const float2* __restrict__ twtab, int twstride) {
  const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const uint32_t mine = smem_u32(sb);
  if constexpr (NS > 1) {
    const int jm = t % NS;
    const int step = jm * (L / (NS * 16)) * twstride;
    float2 w1 = tw_dir<INV>(tw_load<TWS>(twtab, step));
    float2 wr = w1;
#pragma unroll
    for (int r = 1; r < 16; ++r) {
      if ((r & 3) == 0) wr = tw_dir<INV>(tw_load<TWS>(twtab, step * r));
      v[r] = cmul(v[r], wr);
      wr = cmul(wr, w1);
    }
  }
#pragma unroll
  for (int r = 0; r < 16; ++r) sb[spad(16 * t + r)] = v[r];
  __syncwarp();
  float yr[4][4], yi[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int i = 0; i < 4; ++i) yr[q][i] = yi[q][i] = 0.f;
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    // A fragments of F = W16^{kr}: a_i at row k = gid + 8 (i & 1), column
    // r = tig + 4 (i >> 1) of this k-step (inputs 8 ks .. 8 ks + 7)
    uint32_t frh[4], frl[4], fih[4], fil[4], nfih[4], nfil[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = gid + 8 * (i & 1), r = tig + 4 * (i >> 1) + 8 * ks;
      const float2 w = tw_dir<INV>(tw_load<TWS>(twtab, ((k * r) & 15) * (L / 16) * twstride));
      tf32_split<PREC>(w.x, frh[i], frl[i]);
      tf32_split<PREC>(w.y, fih[i], fil[i]);
      nfih[i] = fih[i] ^ 0x80000000u;
      nfil[i] = fil[i] ^ 0x80000000u;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      // B fragments: b0 = U[r = 8 ks + tig][n], b1 = U[r + 4][n], n = gid + 8 q
      const int n = gid + 8 * q;
      const int tn = __shfl_sync(0xffffffffu, t, n);
      const uint32_t an = __shfl_sync(0xffffffffu, mine, n);
      const int r0 = 8 * ks + tig;
      const float2 u0 = lds_f2(an + 8u * (uint32_t)spad(16 * tn + r0));
      const float2 u1 = lds_f2(an + 8u * (uint32_t)spad(16 * tn + r0 + 4));
      uint32_t rh0, rl0, rh1, rl1, ih0, il0, ih1, il1;
      tf32_split<PREC>(u0.x, rh0, rl0);
      tf32_split<PREC>(u1.x, rh1, rl1);
      tf32_split<PREC>(u0.y, ih0, il0);
      tf32_split<PREC>(u1.y, ih1, il1);
      mma_split<PREC>(yr[q], frh, frl, rh0, rh1, rl0, rl1);    // + Fr Ur
      mma_split<PREC>(yr[q], nfih, nfil, ih0, ih1, il0, il1);  // - Fi Ui
      mma_split<PREC>(yi[q], frh, frl, ih0, ih1, il0, il1);    // + Fr Ui
      mma_split<PREC>(yi[q], fih, fil, rh0, rh1, rl0, rl1);    // + Fi Ur
    }
  }
  __syncthreads();  // every warp has read its staged inputs
  // D fragments: d_i at row k = gid + 8 (i >> 1), column n = 2 tig + (i & 1)
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = 2 * tig + h + 8 * q;
      const int tn = __shfl_sync(0xffffffffu, t, n);
      const uint32_t an = __shfl_sync(0xffffffffu, mine, n);
      const int jm = tn % NS;
      const int base = (tn - jm) * 16 + jm;
      sts_f2(an + 8u * (uint32_t)spad(base + gid * NS), make_float2(yr[q][h], yi[q][h]));
      sts_f2(an + 8u * (uint32_t)spad(base + (gid + 8) * NS), make_float2(yr[q][2 + h], yi[q][2 + h]));
    }
  }
}

// ---------------------------------------------------------------- TMA bulk copies
// 1D bulk copies global -> shared (cp.async.bulk) completed on an mbarrier.
// Addresses and sizes must be multiples of 16 bytes.
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make barrier initialisation visible to the async (TMA) proxy
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Bounded wait for phase `phase` of the barrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, int max_tries) {
  for (int i = 0; i < max_tries; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}
// try_wait already suspends for a hardware-chosen interval per attempt; this
// many attempts is far beyond the microseconds a bulk copy takes.
constexpr int WF_WAIT_TRIES = 1 << 20;

// Ampere-style asynchronous copies (16 or 8 bytes per thread) for strided tiles.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// L2 prefetch hint for a contiguous range of bytes (16-byte aligned, a
// multiple of 16, issued in pieces of at most 64 KB).  It changes no data and
// no ordering; a later load of the range hits L2.
__device__ __forceinline__ void prefetch_l2_range(const void* p, size_t bytes) {
  const char* c = static_cast<const char*>(p);
  for (size_t o = 0; o < bytes; o += 65536) {
    const uint32_t n = (uint32_t)(bytes - o < 65536 ? bytes - o : 65536);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + o), "r"(n) : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------- tcgen05 radix-16
// The same radix-16 stage on the 5th-generation tensor cores: each 128-thread
// group of the block is one tcgen05.mma tile whose M = 128 rows are the
// group's transforms (one per thread), with the complex product written as
// one real product of K = N = 32:
//   [Yr | Yi] (128 x 32) = [Ur | Ui] (128 x 32) . G,   G^T (32 x 32) =
//   [[Fr, -Fi], [Fi, Fr]]  (rows: outputs Yr[k], then Yi[k]; columns: Ur[r], Ui[r]),
// TF32 operands in shared memory, FP32 accumulators in tensor memory (TMEM
// lane = row = transform, column = output), read back with tcgen05.ld by
// the thread that owns the transform.  PREC = 3 splits both factors into
// two TF32 parts (lo*hi + hi*lo + hi*hi, small terms first), PREC = 4 takes
// hi*hi alone.  One thread issues the 4 (K = 8 each; 12 for the split) MMAs
// of every tile and commits them to an mbarrier that all threads wait on.
//
// Operand layout (both A and B = G^T, 32 K-values per row, K-major, no
// swizzle): core matrices of 8 rows x 16 bytes, 128 bytes apart along K
// (leading byte offset) and 1024 bytes apart between 8-row groups (stride
// byte offset).

// block state of the tcgen05 stages, set up by the kernel that uses them
struct Tc5Ctx {
  uint32_t a_hi, a_lo;                              // A tiles, 16 KB per 128 threads
  uint32_t b_fwd_hi, b_fwd_lo, b_inv_hi, b_inv_lo;  // G^T, 4 KB each
  uint32_t mbar;                                    // MMA completion barrier
  uint32_t tmem;                                    // TMEM base (lane 0, column 0)
  uint32_t phase;                                   // parity of the next completion
  uint32_t ntiles;
  uint32_t ok;                                      // 0 once a bounded wait gave up
};
__device__ __forceinline__ Tc5Ctx& tc5_ctx() {
  __shared__ Tc5Ctx c;
  return c;
}
// byte offset of element (row, k) in a K-major no-swizzle 32-column operand
__device__ __forceinline__ uint32_t tc5_off(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}
// shared-memory matrix descriptor: start address, leading byte offset 128,
// stride byte offset 1024, the fixed 0b001 at bits 46-48, no swizzle
__device__ __forceinline__ uint64_t tc5_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
         (1ull << 46);
}
// instruction descriptor of kind::tf32: F32 accumulator (bits 4-5 = 1), TF32
// A and B (bits 7-9, 10-12 = 2), both K-major, N = 32 (bits 17-22 = N >> 3),
// M = 128 (bits 24-28 = M >> 4)
constexpr uint32_t kTc5Idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc5_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kTc5Idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc5_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tc5_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc5_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// whole warp: allocate ncols TMEM columns (power of two, >= 32), address to *dst
__device__ __forceinline__ void tc5_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc5_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc5_ld32(uint32_t taddr, float (&y)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) y[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void sts_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
// bounded wait for phase `phase` of an mbarrier given by its shared address
__device__ __forceinline__ bool mbar_wait_addr(uint32_t bar, uint32_t phase, int max_tries) {
  for (int i = 0; i < max_tries; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}

template <int L, int NS, bool INV, bool TWS, int PREC>
__device__ __forceinline__ void tc5_radix16_stage(float2 (&v)[16], float2* sb, int t,
                                                  const float2* __restrict__ twtab, int twstride) {
  Tc5Ctx& cx = tc5_ctx();
  if constexpr (NS > 1) {
    const int jm = t % NS;
    const int step = jm * (L / (NS * 16)) * twstride;
    float2 w1 = tw_dir<INV>(tw_load<TWS>(twtab, step));
    float2 wr = w1;
#pragma unroll
    for (int r = 1; r < 16; ++r) {
      if ((r & 3) == 0) wr = tw_dir<INV>(tw_load<TWS>(twtab, step * r));
      v[r] = cmul(v[r], wr);
      wr = cmul(wr, w1);
    }
  }
  // this thread's transform is row `row` of its group's A tile
  const int tile = threadIdx.x >> 7, row = threadIdx.x & 127;
  const uint32_t ahi = cx.a_hi + (uint32_t)tile * 16384u, alo = cx.a_lo + (uint32_t)tile * 16384u;
#pragma unroll
  for (int kc = 0; kc < 8; ++kc) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 4 * kc + q;
      const float x = k < 16 ? v[k].x : v[k - 16].y;
      tf32_split<PREC == 3 ? 1 : 2>(x, h[q], l[q]);
    }
    sts_v4(ahi + tc5_off(row, 4 * kc), h[0], h[1], h[2], h[3]);
    if constexpr (PREC == 3) sts_v4(alo + tc5_off(row, 4 * kc), l[0], l[1], l[2], l[3]);
  }
  const uint32_t ph = cx.phase;
  fence_async_smem();  // the generic-proxy stores above, seen by the tensor cores
  tc5_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc5_fence_after();
    const uint32_t bhi = INV ? cx.b_inv_hi : cx.b_fwd_hi, blo = INV ? cx.b_inv_lo : cx.b_fwd_lo;
    for (uint32_t tl = 0; tl < cx.ntiles; ++tl) {
      const uint32_t d = cx.tmem + 32u * tl;
      const uint32_t ah = cx.a_hi + tl * 16384u, al = cx.a_lo + tl * 16384u;
      uint32_t acc = 0;
      if constexpr (PREC == 3) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          tc5_mma(d, tc5_desc(al + 256u * s), tc5_desc(bhi + 256u * s), acc);
          acc = 1;
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) tc5_mma(d, tc5_desc(ah + 256u * s), tc5_desc(blo + 256u * s), 1);
      }
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        tc5_mma(d, tc5_desc(ah + 256u * s), tc5_desc(bhi + 256u * s), acc);
        acc = 1;
      }
    }
    tc5_commit(cx.mbar);
  }
  if (!mbar_wait_addr(cx.mbar, ph, WF_WAIT_TRIES)) cx.ok = 0u;
  tc5_fence_after();
  float y[32];
  tc5_ld32(cx.tmem + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16) + 32u * (uint32_t)tile, y);
  tc5_fence_before();
  __syncthreads();  // every thread has passed the wait and read its outputs
  if (threadIdx.x == 0) cx.phase = ph ^ 1u;
  // outputs to their autosort positions, as the FP32 stage stores them
  const int jm = t % NS;
  const int base = (t - jm) * 16 + jm;
#pragma unroll
  for (int k = 0; k < 16; ++k) sb[spad(base + k * NS)] = make_float2(y[k], y[16 + k]);
}

// Block set-up of the tcgen05 stages (every thread calls it): the four G^T
// matrices from the exact twiddle table, the mbarrier, the TMEM columns
// (32 per 128-thread tile, warp 0 allocates), the context.  smem_ab starts a
// region of 1 KB (alignment slack) + (PREC == 3 ? 2 : 1) * 16 KB per tile +
// 16 KB.
template <int L, int PREC>
__device__ __forceinline__ void tc5_setup(unsigned char* smem_ab, uint64_t* mbar, const float2* __restrict__ twtab,
                                          int twstride) {
  Tc5Ctx& cx = tc5_ctx();
  const uint32_t ntiles = blockDim.x / 128;
  const uint32_t abytes = ntiles * 16384u;
  const uint32_t base = (smem_u32(smem_ab) + 1023u) & ~1023u;  // 1 KB slack reserved
  const uint32_t bbase = base + abytes * (PREC == 3 ? 2u : 1u);
  for (int i = threadIdx.x; i < 4 * 32 * 32; i += blockDim.x) {
    const int mat = i >> 10, j = (i >> 5) & 31, kk = i & 31;  // mat: fwd hi, fwd lo, inv hi, inv lo
    const bool inv = mat >= 2;
    const int k = j & 15, r = kk & 15;
    float2 w = twtab[((k * r) & 15) * (L / 16) * twstride];
    if (inv) w.y = -w.y;
    // rows j < 16: Yr[k] = Fr Ur - Fi Ui; rows j >= 16: Yi[k] = Fi Ur + Fr Ui
    const float g = (j < 16) ? (kk < 16 ? w.x : -w.y) : (kk < 16 ? w.y : w.x);
    uint32_t hi, lo;
    tf32_split<1>(g, hi, lo);
    const uint32_t addr = bbase + (uint32_t)(mat >> 1) * 8192u + (uint32_t)(mat & 1) * 4096u + tc5_off(j, kk);
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"((mat & 1) ? lo : hi) : "memory");
  }
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    mbar_fence_init();
    cx.a_hi = base;
    cx.a_lo = base + abytes;
    cx.b_fwd_hi = bbase;
    cx.b_fwd_lo = bbase + 4096u;
    cx.b_inv_hi = bbase + 8192u;
    cx.b_inv_lo = bbase + 12288u;
    cx.mbar = smem_u32(mbar);
    cx.phase = 0u;
    cx.ntiles = ntiles;
    cx.ok = 1u;
  }
  if (threadIdx.x < 32) tc5_alloc(smem_u32(&cx.tmem), 32u * ntiles);
  fence_async_smem();
  tc5_fence_before();
  __syncthreads();
  tc5_fence_after();
}

// Release the TMEM columns (every thread calls it, after its last tcgen05.ld).
__device__ __forceinline__ void tc5_teardown() {
  Tc5Ctx& cx = tc5_ctx();
  tc5_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc5_fence_after();
    tc5_dealloc(cx.tmem, 32u * cx.ntiles);
  }
}

// One Stockham autosort stage (radix R, sub-transform length NS) of a
// length-L complex DFT computed by TPF = L/E threads, E values per thread.
// Inputs are the "natural" layout (thread t holds x[t + m*TPF], m =
// b + r*(E/R)); outputs go to shared memory at their autosort positions, or,
// for the last stage, back to the registers in the natural layout.
// twtab holds exp(-2 pi i k / (L*twstride)), k < L*twstride.  PREC != 0 runs
// the radix-16 stages of 16-value threads on the tensor cores (above).
template <int L, int E, int NS, bool INV, bool WARP, bool TWS = false, int PREC = 0>
struct FFTStages {
  static __device__ __forceinline__ void run(float2 (&v)[E], float2* sb, int t,
                                             const float2* __restrict__ twtab, int twstride) {
    constexpr int R = StageRadix<L, E, NS>::value;
    constexpr int TPF = L / E;
    constexpr bool LAST = (NS * R == L);
    constexpr bool TC = (PREC != 0 && R == 16 && E == 16 && !WARP);
    if constexpr (TC) {
      if constexpr (PREC >= 3) tc5_radix16_stage<L, NS, INV, TWS, PREC>(v, sb, t, twtab, twstride);
      else tc_radix16_stage<L, NS, INV, TWS, PREC>(v, sb, t, twtab, twstride);
      fft_sync<WARP>();
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = sb[spad(t + m * TPF)];
      fft_sync<WARP>();
      if constexpr (!LAST) FFTStages<L, E, NS * R, INV, WARP, TWS, PREC>::run(v, sb, t, twtab, twstride);
    } else {
      stage_fp32(v, sb, t, twtab, twstride);
    }
  }

  static __device__ __forceinline__ void stage_fp32(float2 (&v)[E], float2* sb, int t,
                                                    const float2* __restrict__ twtab, int twstride) {
    constexpr int R = StageRadix<L, E, NS>::value;
    constexpr int TPF = L / E;
    constexpr int B = E / R;
    constexpr bool LAST = (NS * R == L);
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = t + b * TPF;
      const int jm = j % NS;
      float2 u[R];
#pragma unroll
      for (int r = 0; r < R; ++r) u[r] = v[b + r * B];
      if constexpr (NS > 1) {
        // twiddles W_{NS R}^{jm r}: exact table values every 4th power,
        // products in between (at most 3 multiplications deep)
        const int step = jm * (L / (NS * R)) * twstride;
        float2 w1 = tw_dir<INV>(tw_load<TWS>(twtab, step));
        float2 wr = w1;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          if ((r & 3) == 0) wr = tw_dir<INV>(tw_load<TWS>(twtab, step * r));
          u[r] = cmul(u[r], wr);
          wr = cmul(wr, w1);
        }
      }
      dftR<R, INV>(u);
      if constexpr (LAST) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[b + r * B] = u[r];
      } else {
        const int base = (j - jm) * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) sb[spad(base + r * NS)] = u[r];
      }
    }
    if constexpr (!LAST) {
      fft_sync<WARP>();
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = sb[spad(t + m * TPF)];
      fft_sync<WARP>();
      FFTStages<L, E, NS * R, INV, WARP, TWS, PREC>::run(v, sb, t, twtab, twstride);
    }
  }
};

// Full complex DFT of length L (no scaling).  Every thread of the block (or
// of the warp, WARP = true) must call it; sb is this transform's own padded
// shared buffer of SPad<L>::size values.
template <int L, int E, bool INV, bool WARP = false, bool TWS = false, int PREC = 0>
__device__ __forceinline__ void fft_block(float2 (&v)[E], float2* sb, int t,
                                          const float2* __restrict__ twtab, int twstride) {
  FFTStages<L, E, 1, INV, WARP, TWS, PREC>::run(v, sb, t, twtab, twstride);
}

// W_N^k (N = 2M) for the k = t + m*(M/E) a thread handles in c2r_pre and
// r2c_post; loaded once, early, and passed to both.
template <int M, int E>
__device__ __forceinline__ void load_rtw(float2 (&wk)[E], int t, const float2* __restrict__ twx) {
  constexpr int TPF = M / E;
#pragma unroll
  for (int m = 0; m < E; ++m) wk[m] = __ldg(&twx[t + m * TPF]);
}

// ---------------------------------------------------------------- real rows
// Real length-N rows (N = 2M) through complex length-M transforms:
// z[n] = x[2n] + i x[2n+1].  The packed half spectrum holds X[k] at k = 1..M-1
// and (X[0], X[M]) -- both real -- as the pair in slot 0.

// Before an inverse complex FFT: X (natural layout in v) -> Z so that
// IFFT_M(Z) / M gives z.  Here the 1/N scaling of the inverse real DFT is
// folded in.  twx = exp(-2 pi i k / N).
template <int M, int E, bool WARP = false>
__device__ __forceinline__ void c2r_pre_w(float2 (&v)[E], float2* sb, int t, const float2 (&wk)[E]) {
  constexpr int TPF = M / E;
  const float s = 0.5f / (float)M;
#pragma unroll
  for (int m = 0; m < E; ++m) sb[spad(t + m * TPF)] = v[m];
  fft_sync<WARP>();
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int k = t + m * TPF;
    float2 X = v[m];
    if (k == 0) {
      v[m] = make_float2((X.x + X.y) * s, (X.x - X.y) * s);
    } else {
      float2 Xm = cconj(sb[spad(M - k)]);
      float2 Ek = cadd(X, Xm);
      float2 Ok = cmul(csub(X, Xm), cconj(wk[m]));
      v[m] = make_float2((Ek.x - Ok.y) * s, (Ek.y + Ok.x) * s);
    }
  }
  fft_sync<WARP>();
}

template <int M, int E, bool WARP = false>
__device__ __forceinline__ void r2c_post_w(float2 (&v)[E], float2* sb, int t, const float2 (&wk)[E]) {
  constexpr int TPF = M / E;
#pragma unroll
  for (int m = 0; m < E; ++m) sb[spad(t + m * TPF)] = v[m];
  fft_sync<WARP>();
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int k = t + m * TPF;
    float2 Z = v[m];
    if (k == 0) {
      v[m] = make_float2(Z.x + Z.y, Z.x - Z.y);
    } else {
      float2 Zm = cconj(sb[spad(M - k)]);
      float2 Ek = cscale(cadd(Z, Zm), 0.5f);
      float2 D = cscale(csub(Z, Zm), 0.5f);
      float2 Ok = make_float2(D.y, -D.x);
      v[m] = cadd(Ek, cmul(wk[m], Ok));
    }
  }
  fft_sync<WARP>();
}

template <int M, int E, bool WARP = false>
__device__ __forceinline__ void c2r_pre(float2 (&v)[E], float2* sb, int t,
                                        const float2* __restrict__ twx) {
  constexpr int TPF = M / E;
  const float s = 0.5f / (float)M;  // 1/(2M) = 1/N, times the 1/2 of E and O
#pragma unroll
  for (int m = 0; m < E; ++m) sb[spad(t + m * TPF)] = v[m];
  fft_sync<WARP>();
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int k = t + m * TPF;
    float2 X = v[m];
    if (k == 0) {
      v[m] = make_float2((X.x + X.y) * s * 1.0f, (X.x - X.y) * s);
    } else {
      float2 Xm = cconj(sb[spad(M - k)]);
      float2 Ek = cadd(X, Xm);
      float2 Ok = cmul(csub(X, Xm), cconj(__ldg(&twx[k])));
      // Z = E + i O
      v[m] = make_float2((Ek.x - Ok.y) * s, (Ek.y + Ok.x) * s);
    }
  }
  fft_sync<WARP>();
}

// After a forward complex FFT: Z (natural layout) -> packed X.
template <int M, int E, bool WARP = false>
__device__ __forceinline__ void r2c_post(float2 (&v)[E], float2* sb, int t,
                                         const float2* __restrict__ twx) {
  constexpr int TPF = M / E;
#pragma unroll
  for (int m = 0; m < E; ++m) sb[spad(t + m * TPF)] = v[m];
  fft_sync<WARP>();
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int k = t + m * TPF;
    float2 Z = v[m];
    if (k == 0) {
      v[m] = make_float2(Z.x + Z.y, Z.x - Z.y);
    } else {
      float2 Zm = cconj(sb[spad(M - k)]);
      float2 Ek = cscale(cadd(Z, Zm), 0.5f);
      float2 D = cscale(csub(Z, Zm), 0.5f);
      float2 Ok = make_float2(D.y, -D.x);  // D / i
      v[m] = cadd(Ek, cmul(__ldg(&twx[k]), Ok));
    }
  }
  fft_sync<WARP>();
}

// ---------------------------------------------------------------- state
// Device-resident solver state.  Problem constants are written by the setup
// kernels; lambda and the derived messenger covariances by the controller.
struct WfState {
  // problem constants
  double tau[3];      // tau_i for parts 2DF, RF, PX (0 when absent)
  double off[3];      // Nbar_i = (given eigenvalue) + off_i  (moved white - tau)
  double var_shift;   // N_PX used for the residual: nbar_px - off[2]
  double du2;         // ||d_unmasked||^2
  double min_v, min_f, min_s, min_a2;
  unsigned err;       // setup validation bits (WF_ERR_*)
  int n_unmasked;
  // cooling / control
  double lam;         // current lambda
  float Tf[3];        // lambda * tau_i as float
  float T0s[2];       // T_0 with which the stored t_0 was made, by parity slot
  double prev_rho2;   // adaptive rule reference (< 0: none)
  double rho2, gm2, g2, rel_u, rel_m;
  int done;           // 1: stop (converged or out of iterations)
  int status;         // 0 converged, 3 out of iterations, 4 stalled
  int iter;           // iterations completed in this run
  int checkpoints;
  int level, in_level;
  int stall_n;        // checkpoints at lambda = 1 without a 1% drop of rho2
  int skip_resid;     // 1: the next checkpoint's residual is not needed (fixed
                      // schedule above lambda = 1, not the last checkpoint)
  double stall_ref;   // rho2 those checkpoints are measured against (<= 0: none)
};

enum : unsigned {
  WF_ERR_D_NONFINITE = 1u, WF_ERR_VAR = 2u, WF_ERR_C = 4u, WF_ERR_P1F = 8u,
  WF_ERR_PST = 16u, WF_ERR_A2 = 32u, WF_ERR_ASYM = 64u, WF_ERR_ALLMASKED = 128u,
  WF_ERR_TIMEOUT = 256u  // a bounded wait on a bulk copy gave up (never expected)
};

// Every messenger update has the form x = (B a + A b)/(A + B): the mean of x
// under the Gaussian terms (x-a)^2/A + (x-b)^2/B, i.e. the
// (A^-1 + B^-1)^-1 (A^-1 a + B^-1 b) of eqs. (ew_t), (2mess_t1)-(2mess_t0).
__device__ __forceinline__ float link_w(float A, float B) { return __fdividef(B, A + B); }

// ---------------------------------------------------------------- grid barrier
// (for cooperative launches whose CTAs are all resident: the one-launch sweep
// of wf_fused.cu and the persistent batch of wf_batchk.cu)
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Waits this many polls at most (each a global load, about half a
// microsecond); a sweep's barrier normally waits one or two microseconds.
constexpr int WF_GRID_TRIES = 1 << 21;

// All CTAs of the grid meet here.  bar[0] counts the arrivals of this launch
// (zeroed before it starts); the k-th barrier of the launch is passed once
// it reaches k * nblocks.  Each arrival is an acquire-release add (the CTA's
// writes, ordered before it by the block barrier, are released; the last
// arrival need not wait for a second word to change), and the waits are
// acquire loads of the same word, so one round trip to L2 separates the
// last arrival from the others' release.  bar[2] is the abort word.
// Returns false, for every thread of the CTA, if the wait gave up or
// another CTA aborted.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int* ok_s, unsigned* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned seen;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(seen) : "l"(bar) : "memory");
    for (int i = 0; seen + 1u < target; ++i) {
      if (i >= WF_GRID_TRIES || ld_relaxed_gpu(&bar[2]) != 0u) {
        atomicExch(&bar[2], 1u);
        atomicOr(err, WF_ERR_TIMEOUT);
        ok = 0;
        break;
      }
      seen = ld_acquire_gpu(bar) - 1u;
    }
    *ok_s = ok;
  }
  __syncthreads();
  return *ok_s != 0;
}


}  // namespace wf
