#pragma once
// Device code of the fused per-cell kernels of the fast spectral collision operator
// (sm_103a), shared by the kernel translation units collide_f32.cu, collide_f64.cu,
// collide_tc.cu and collide_2d.cu.
//
// Paper: arxiv 1608.08009.  Per cell (Sec. 4.2): one forward 3D transform of f
// (Eq. FC), then for every separated quadrature term j the coefficients
// (alpha_j + i alpha'_j) fhat and one inverse 3D transform (Eq. FU) whose real and
// imaginary parts are the two factors of the gain term (Sec. 3.3, decoupling formula),
// accumulated as Q+ += w_j Re Im; then the loss term L = inverse(D fhat), Q = Q+ - f L,
// the conservation projection (Sec. 3.2, Eq. minim1) and optionally the collision step
// f <- f + dt Q (Eq. f_coll), all in one launch: f is read once and Q (or the new f)
// written once per cell.
//
// Work decomposition.  A cell is owned by a thread-block cluster of C CTAs.
//  * Spectrum: CTA c keeps fhat(kx, ky, kz) for the ky-slab [c N/C, (c+1) N/C), all kx
//    and kz: in registers (float32, thread (ky, kz) holds its kx pencil) or shared memory.
//  * Physical space: CTA q owns the x-slab [q N/C, (q+1) N/C); the gain accumulator of
//    its points lives in registers (thread (x, z) holds the N values along y).
//  * One inverse 3D transform = pass along kx (pencils of the CTA's ky-slab, in
//    registers) whose N outputs are scattered by x into the owners' shared memory through
//    distributed shared memory, a cluster barrier, then the passes along kz and ky inside
//    each x-plane of the owner.
//  * Every 1D pass is a fully unrolled radix-4/2 FFT of one pencil held by one thread.
// Twiddles, kernel tables and weights are float32 for the BOLTZ_FP32_FFT path and
// float64 for BOLTZ_FP64.  Moments, projection and the update are float64 in both.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <string>

#include "fft_regs.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace boltz {

// Device status word of this translation unit (each unit has its own copy; the host
// reads and clears all of them): bit 0 non-finite output, bit 2 bad cell index, bit 3
// a bounded tensor-core wait gave up.
static __device__ unsigned int g_boltz_status;

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

template <typename T> __device__ __forceinline__ typename Vec2<T>::type mk2(T a, T b);
template <> __device__ __forceinline__ float2 mk2<float>(float a, float b) { return make_float2(a, b); }
template <> __device__ __forceinline__ double2 mk2<double>(double a, double b) { return make_double2(a, b); }

// CollideArgs (internal.h) is the argument block of every collision kernel.


// Status bits of g_boltz_status.
constexpr unsigned kStatusNonFinite = 1u;
constexpr unsigned kStatusBadIndex = 4u;
constexpr unsigned kStatusTimeout = 8u;  // a bounded wait on an mbarrier gave up

// Tensor memory budget.  tcgen05.alloc waits while the SM lacks a free, aligned block of
// the requested columns, and a CTA that waits there while cluster peers on other SMs wait
// for it (at a cluster barrier, holding their own columns) could close a cycle with the
// CTAs of another kernel running on another stream.  So no allocation may ever wait:
// every kernel that shares its SM allocates in shares of exactly kTmemShare columns (one
// size, so the 512 columns never fragment; a CTA may hold a few) and takes enough shared
// memory per share that at most 8 shares fit on an SM (8 x 64 = 512 columns); a kernel
// that needs one larger allocation takes enough shared memory that no share fits beside
// it.  tmem_launch_smem (host side, below) sizes both from the device's own
// shared-memory attributes.
constexpr int kTmemShare = 64;

// Tensor-core transform modes of the float32 path (0: register FFT).
constexpr int kTcNone = 0, kTcTF32 = 1, kTc3xBF16 = 2, kTc3xTF32 = 3;

template <typename T, int N, int C, int TC = kTcNone>
struct CollideCfg {
  static constexpr int NP = N / C;          // slab width (x for physical, ky for spectral)
  static constexpr int THREADS = NP * N;    // one pencil per thread in every pass
  static constexpr int WARPS = THREADS / 32;
  // CTAs per SM asked of the register allocator.  float32 32^3 with C = 8: 4 (128
  // registers; the spectrum pencil is in TMEM and the x-plane buffer single, 34 KB of
  // shared memory): sixteen warps per SM hide the table loads and barrier waits.  On
  // GB300: 2 CTAs (252 registers) 131k, 3 CTAs (168 registers, double buffer) 147k,
  // 4 CTAs 161k cell-collisions/s.
  // The same single-buffer layout serves C = 4 (256-thread CTAs, two per SM) and C = 16
  // (64-thread CTAs, eight per SM).
  static constexpr bool kQuad = (sizeof(T) == 4 && N == 32 && (C == 4 || C == 8 || C == 16) && TC == kTcNone);
  // float64 32^3 with the spectrum in TMEM: two CTAs per SM (at most 256 registers)
  static constexpr int MIN_BLOCKS = (TC == kTcTF32 || TC == kTc3xBF16) ? 2
                                    : (TC == kTc3xTF32)                  ? 1
                                    : kQuad                              ? C / 2
                                    : (sizeof(T) == 8 && N == 32)        ? 2
                                                                         : 1;
  using T2 = typename Vec2<T>::type;
  static constexpr bool kF32 = sizeof(T) == 4;
  // float32: the spectrum pencil of each thread is private to it (TMEM at N = 16, 32,
  // registers otherwise) and the x-plane buffer is double-buffered (one cluster barrier
  // per term) except in the 4-CTA 32^3 configuration, which trades the second buffer for
  // occupancy; float64 (register bound) keeps a single x-plane buffer.
  static constexpr bool kRegSpec = kF32;
  static constexpr int NXB = (kRegSpec && TC == kTcNone && !kQuad) ? 2 : 1;
  // Register-FFT paths at N = 16, 32 (float64: 32 only): the spectrum pencil of each
  // thread lives in TMEM (warp w: lanes 32 (w % 4) .., column group w / 4) instead of
  // registers (float32) or a shared-memory slab (float64, which then fits two CTAs per SM
  // at 32^3; at 16^3 the slab is small and TMEM measured no faster).  A group of four
  // warps takes GROUP_COLS columns: the N real parts, then the N imaginary parts, CPV
  // 32-bit columns per value (a float64 value is its low and high words).
  static constexpr bool kTmemSpec = TC == kTcNone && N % 16 == 0 && (kF32 || N == 32);
  static constexpr int CPV = (int)(sizeof(T) / 4);
  static constexpr int GROUP_COLS = 2 * N * CPV;
  static constexpr int TMEM_NEED = ((THREADS / 32 + 3) / 4) * GROUP_COLS;
  static constexpr int TMEM_COLS = TMEM_NEED <= 64 ? 64 : TMEM_NEED <= 128 ? 128 : TMEM_NEED <= 256 ? 256 : 512;
  // The spectrum's columns as kTmemShare-column allocations: one when they all fit in
  // one, otherwise SPG = GROUP_COLS / kTmemShare per group of four warps (SPG = 1: real
  // and imaginary halves in one share; SPG = 2: one share each).
  static constexpr int SPG = GROUP_COLS <= kTmemShare ? 1 : GROUP_COLS / kTmemShare;
  static constexpr int TMEM_SHARES = !kTmemSpec ? 0 : TMEM_NEED <= kTmemShare ? 1 : ((THREADS / 32 + 3) / 4) * SPG;
  static_assert(!kTmemSpec || TMEM_SHARES <= 4, "spectrum shares per CTA");
  static_assert(!kTmemSpec || TMEM_SHARES == 1 || (SPG == 1 && GROUP_COLS <= kTmemShare) ||
                    (SPG == 2 && GROUP_COLS == 2 * kTmemShare),
                "whole shares per warp group");
  // x-plane buffer: the NP x-values of a slab are grouped in chunks of VEC (16 bytes:
  // two float2 or one double2); element (xl, ky, k) (k = kz or z) sits at
  // ((xl / VEC) N + ky) RW VEC + k VEC + xl % VEC.  A warp of the kx pass (lanes along
  // kz) then stores 32 contiguous 16-byte chunks to a peer: full 32-byte sectors on the
  // SM-to-SM network.  RW = N + 1 (odd) keeps the in-plane passes conflict-free with lanes
  // ordered (x % VEC, ky) and (x % VEC, z).
  static constexpr int VEC = kF32 ? 2 : 1;
  static constexpr int NCH = NP / VEC;  // chunks per (ky, k)
  static constexpr int RW = N + 1;
  static constexpr size_t FH = (kRegSpec || kTmemSpec) ? 0 : (size_t)N * NP * N;  // spectrum slab [kx][kyl][kz]
  static constexpr size_t XB = (size_t)NCH * N * RW * VEC;
  static constexpr size_t OFF_XB = FH * sizeof(T2);
  static constexpr size_t OFF_RED = OFF_XB + NXB * XB * sizeof(T2);
  // red: [WARPS][5] warp partials, then [5] Phi g and [5] Phi f_in of this CTA; then
  // the last-arrival flag of split launches, room for four scatter mbarriers and four
  // TMEM addresses (the spectrum's allocations)
  static constexpr size_t OFF_FLAG = OFF_RED + (size_t)(WARPS + 2) * 5 * sizeof(double);
  static constexpr size_t OFF_MBAR = OFF_FLAG + 16;
  static constexpr size_t OFF_TSLOT = OFF_MBAR + 32;
  // tensor-core transforms: operand tiles (rows of 2N floats, K-major without swizzle:
  // 8-row x 16-byte core matrices, K-adjacent ones 128 bytes apart), the DFT matrix,
  // the MMA-completion barrier and the TMEM address
  static constexpr int TC_K = 2 * N;
  static constexpr int TC_SPLIT = (TC == kTc3xTF32 || TC == kTc3xBF16) ? 2 : 1;
  static constexpr int TC_ES = (TC == kTc3xBF16) ? 2 : 4;  // operand element bytes
  static constexpr size_t OFF_TCA = (OFF_TSLOT + 16 + 1023) / 1024 * 1024;
  static constexpr size_t TCA_BYTES = (TC != kTcNone) ? (size_t)TC_SPLIT * THREADS * TC_K * TC_ES : 0;
  static constexpr size_t OFF_TCW = OFF_TCA + TCA_BYTES;
  static constexpr size_t TCW_BYTES = (TC != kTcNone) ? (size_t)TC_SPLIT * TC_K * TC_K * TC_ES : 0;
  static constexpr size_t OFF_TCB = OFF_TCW + TCW_BYTES;  // mbarrier (8 B) + TMEM address (4 B)
  // 32^3 single-buffer configurations: the kx-pass scatter uses st.async, which signals
  // the owner's mbarrier (at OFF_MBAR) with the bytes it delivers
  static constexpr bool kAsyncScatter = kQuad && C > 1;
  static constexpr uint32_t SCATTER_BYTES = (uint32_t)NP * N * N * 2 * sizeof(T);  // received per term
  static_assert(!kAsyncScatter || (NCH <= 4 && (THREADS / NCH) % 32 == 0), "per-chunk mbarriers and barriers");
  static constexpr size_t SMEM = (TC != kTcNone) ? OFF_TCB + 16 : OFF_TSLOT + 16;
  // TMEM columns held: the spectrum pencils, or the tensor-core accumulator (2N <= 64)
  static constexpr int TC_TMEM_COLS = kTmemShare;
  static constexpr int TMEM_HELD = kTmemSpec ? TMEM_SHARES * kTmemShare : (TC != kTcNone) ? TC_TMEM_COLS : 0;
  static_assert(TC == kTcNone || (kF32 && THREADS == 128), "tensor-core transforms: float32, 128 pencils per CTA");
  static_assert(TC == kTcNone || 2 * N <= TC_TMEM_COLS, "tensor-core accumulator fits its columns");
  static_assert(THREADS % 32 == 0, "whole warps");
  static_assert(NP % VEC == 0, "whole chunks");
  static_assert(OFF_XB % 16 == 0 && (XB * sizeof(T2)) % 16 == 0, "16-byte aligned buffers");
  static_assert(SMEM <= 232448, "shared memory per CTA");
  static __device__ __forceinline__ int elem(int xl, int ky, int k) {
    return ((xl / VEC) * N + ky) * RW * VEC + k * VEC + xl % VEC;
  }
};

template <int C>
__device__ __forceinline__ void cluster_barrier() {
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
}

// Cluster barrier that separates this CTA's reads of its own shared memory from the
// peers' next writes into it (write-after-read).  The arrive keeps its default .release
// semantics: by the PTX memory model that orders every shared-memory load issued before
// it ahead of any store a peer makes after its matching wait, whatever the compiler and
// the hardware do with the loads' consumers.  (A relaxed arrive would rely on the loads
// having completed when the arrive issues, which nothing guarantees.)
template <int C>
__device__ __forceinline__ void cluster_barrier_war() {
  if constexpr (C > 1) {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  } else {
    __syncthreads();
  }
}

// The two halves of cluster_barrier_war (C > 1), for a caller with work that touches
// neither side of the hazard between them: the arrive right after the last read, the
// wait right before the first store into a peer.
template <int C>
__device__ __forceinline__ void cluster_arrive_war() {
  static_assert(C > 1, "cluster only");
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
template <int C>
__device__ __forceinline__ void cluster_wait_war() {
  static_assert(C > 1, "cluster only");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int C, typename P>
__device__ __forceinline__ P* cta_smem(P* p, int r) {
  if constexpr (C > 1) {
    return cg::this_cluster().map_shared_rank(p, (unsigned)r);
  } else {
    return p;
  }
}

// float -> double by moving the IEEE 754 fields on the integer pipes (binary32 to
// binary64: exponent rebiased by 1023 - 127 = 896, fraction shifted left by 29;
// subnormals normalised with a leading-zero count; zeros, infinities and NaNs keep their
// class).  Exact, like the hardware conversion, which on GB300 issues to the FP64 pipe
// (1/64 of the FP32 rate).  Used where that pipe binds (the 2D kernel); in the 3D
// kernels, bound by latency and issue instead, the extra integer instructions measured
// slower and the hardware conversion stays.
template <typename X>
__device__ __forceinline__ double to_f64(X x) {
  return (double)x;
}
template <>
__device__ __forceinline__ double to_f64<float>(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t e = (u >> 23) & 0xffu, s = u & 0x80000000u;
  uint32_t hi = s | (((u & 0x7fffffffu) >> 3) + 0x38000000u), lo = u << 29;
  if (e == 0xffu) hi |= 0x7ff00000u;  // infinity / NaN: all-ones exponent
  if (e == 0u) {
    const uint32_t m = u & 0x7fffffu;
    if (m == 0u) {
      hi = s;
      lo = 0u;
    } else {  // subnormal m 2^-149: normalise to 1.f 2^(-126 - sh)
      const int sh = __clz((int)m) - 8;
      const uint32_t mn = m << sh;
      hi = s | ((uint32_t)(897 - sh) << 20) | ((mn & 0x7fffffu) >> 3);
      lo = mn << 29;
    }
  }
  return __hiloint2double((int)hi, (int)lo);
}

// double -> float, rounded to nearest (ties to even), on the integer pipes for results in
// the normal float range: the 23 fraction bits are the top of the double's 52, the 29
// dropped bits decide the rounding, and a carry out of the fraction steps the exponent
// (up to infinity, as the rounding requires).  Zeros, float subnormals, overflow,
// infinities and NaNs take the hardware conversion.
template <typename X>
__device__ __forceinline__ X from_f64(double d) {
  return (X)d;
}
template <>
__device__ __forceinline__ float from_f64<float>(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;  // float biased exponent
  if (e < 1 || e > 254) return (float)d;
  uint32_t r = (hi & 0x80000000u) | ((uint32_t)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rem = lo & 0x1fffffffu, half = 0x10000000u;
  r += (rem > half || (rem == half && (r & 1u))) ? 1u : 0u;
  return __uint_as_float(r);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared::cluster address of `addr` (a shared::cta address) in the CTA of rank r
__device__ __forceinline__ uint32_t cluster_addr(uint32_t addr, uint32_t r) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(addr), "r"(r));
  return out;
}

// One 16-byte chunk of the x-plane buffer: two float2 (x, x + 1) or one double2.
__device__ __forceinline__ void st_cluster_chunk(uint32_t a, const float* re, const float* im) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};"
               :: "r"(a), "f"(re[0]), "f"(im[0]), "f"(re[1]), "f"(im[1]) : "memory");
}
__device__ __forceinline__ void st_cluster_chunk(uint32_t a, const double* re, const double* im) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" :: "r"(a), "d"(re[0]), "d"(im[0]) : "memory");
}
// One 16-byte chunk to a peer's shared memory with st.async: the store completes a
// transaction of 16 bytes on the peer's mbarrier (both addresses shared::cluster).
__device__ __forceinline__ void st_async_chunk(uint32_t a, const float* re, const float* im, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
               :: "r"(a), "f"(re[0]), "f"(im[0]), "f"(re[1]), "f"(im[1]), "r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
}
// Bounded wait for the phase with parity `phase` of a local mbarrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 20) && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
  }
  return done != 0;
}
__device__ __forceinline__ void ld_cluster_chunk(uint32_t a, float* re, float* im) {
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(re[0]), "=f"(im[0]), "=f"(re[1]), "=f"(im[1]) : "r"(a) : "memory");
}
__device__ __forceinline__ void ld_cluster_chunk(uint32_t a, double* re, double* im) {
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(re[0]), "=d"(im[0]) : "r"(a) : "memory");
}
__device__ __forceinline__ void st_local_chunk(float2* p, const float* re, const float* im) {
  *reinterpret_cast<float4*>(p) = make_float4(re[0], im[0], re[1], im[1]);
}
__device__ __forceinline__ void st_local_chunk(double2* p, const double* re, const double* im) {
  *p = make_double2(re[0], im[0]);
}
__device__ __forceinline__ void ld_local_chunk(const float2* p, float* re, float* im) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  re[0] = v.x; im[0] = v.y; re[1] = v.z; im[1] = v.w;
}
__device__ __forceinline__ void ld_local_chunk(const double2* p, double* re, double* im) {
  const double2 v = *p;
  re[0] = v.x; im[0] = v.y;
}

// Values of launch cell `cell` that the thread of velocity-x index x loads: the cell
// itself, or with the transport stage fused in (CollideArgs::tr) the cell the shifted
// interval comes from, or the boundary state beyond the row's end.
template <typename TIO>
__device__ __forceinline__ const TIO* cell_input(const CollideArgs& a, long long cell, int x, long long n) {
  if (a.tr.nx <= 0) return reinterpret_cast<const TIO*>(a.f_in) + cell * n;
  const long long row = cell / a.tr.nx, j = cell % a.tr.nx;
  const long long src = j - ((long long)((a.tr.shift_pos >> x) & 1ull) - (long long)((a.tr.shift_neg >> x) & 1ull));
  if (src < 0) return reinterpret_cast<const TIO*>(a.tr.inflow_lo) + row * n;
  if (src >= a.tr.nx) return reinterpret_cast<const TIO*>(a.tr.inflow_hi) + row * n;
  return reinterpret_cast<const TIO*>(a.f_in) + (row * a.tr.nx + src) * n;
}

// Term-group scratch of launch cell lc: partial gains [G][n], loss multipliers [n] and
// the cell's arrival count, by launch position or through the block index of
// CollideArgs::split_idx.
template <typename T>
__device__ __forceinline__ void split_scratch(const CollideArgs& args, long long lc, int G, int n, T*& part,
                                              T*& lossp, unsigned*& arr) {
  if (args.split_idx) {
    char* blk = static_cast<char*>(args.part) + (size_t)args.split_idx[lc] * args.split_unit;
    part = reinterpret_cast<T*>(blk);
    lossp = part + (size_t)G * n;
    arr = reinterpret_cast<unsigned*>(lossp + n);
  } else {
    part = reinterpret_cast<T*>(args.part) + (size_t)lc * G * n;
    lossp = reinterpret_cast<T*>(args.loss) + (size_t)lc * n;
    arr = args.arrivals + lc;
  }
}

// Projection of Sec. 3.2 (Eq. minim1) for one cell owned by a cluster: m[5] is this
// thread's share of Phi g; red holds [WARPS][5] scratch, then [5] Phi g and [5] Phi f_in
// (the targets, when computed) of this CTA.  Returns c5 = G (U - Phi g), zero without
// projection; U is Phi f_in (compute_targets), Utgt[cell] or zero.  Ends with a cluster
// barrier, after which no CTA reads a peer's shared memory.
template <int C, int WARPS>
__device__ __forceinline__ void cluster_correction(const CollideArgs& args, const double (&m)[5], double* red,
                                                   long long cell, bool writable, int rank, int t,
                                                   double (&c5)[5]) {
  const int lane = t & 31, warp = t >> 5;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const double s = warp_sum(m[r]);
    if (lane == 0) red[warp * 5 + r] = s;
  }
  __syncthreads();
  if (t < 5) {
    double s = 0.0;
    for (int w = 0; w < WARPS; ++w) s += red[w * 5 + t];
    red[WARPS * 5 + t] = s;  // this CTA's partial sums
  }
  cluster_barrier<C>();
#pragma unroll
  for (int r = 0; r < 5; ++r) c5[r] = 0.0;
  if (args.project) {
    double tot[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, tgt[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < C; ++q) {
      const double* p = cta_smem<C>(red + WARPS * 5, q);
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        tot[r] += p[r];
        if (args.compute_targets) tgt[r] += p[5 + r];
      }
    }
    if (!args.compute_targets && args.Utgt) {
#pragma unroll
      for (int r = 0; r < 5; ++r) tgt[r] = args.Utgt[cell * 5 + r];
    }
    if (args.compute_targets && args.Utgt && writable && rank == 0) {
#pragma unroll
      for (int r = 0; r < 5; ++r)
        if (t == r) args.Utgt[cell * 5 + r] = tgt[r];  // constant register index
    }
    double rhs[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) rhs[r] = tgt[r] - tot[r];
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 5; ++k) s += args.geom.G[r * 5 + k] * rhs[k];
      c5[r] = s;
    }
  }
  cluster_barrier<C>();  // no CTA leaves while a peer may still read its partial sums
}

// 16 consecutive 32-bit TMEM columns of this thread's lane <-> registers (tcgen05 32x32b)
__device__ __forceinline__ void tmem_st16(uint32_t addr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          addr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t addr, float* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]),
        "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
      : "r"(addr)
      : "memory");
}

// tcgen05.wait::ld with the 16 destination registers of an earlier tcgen05.ld as in-out
// operands.  The registers of a TMEM load hold their values only once the wait has
// completed, and a plain wait orders memory operations alone: arithmetic that reads the
// registers could be scheduled above it.  Tied to the wait, every reader depends on it.
// The first wait blocks until all of the thread's loads have completed; the ones after it
// only tie their registers.
__device__ __forceinline__ void tmem_wait_ld16(float* v) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]),
                 "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]), "+f"(v[15])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld16(uint32_t* v) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                 "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld32(float* v) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]),
                 "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]), "+f"(v[15]),
                 "+f"(v[16]), "+f"(v[17]), "+f"(v[18]), "+f"(v[19]), "+f"(v[20]), "+f"(v[21]), "+f"(v[22]), "+f"(v[23]),
                 "+f"(v[24]), "+f"(v[25]), "+f"(v[26]), "+f"(v[27]), "+f"(v[28]), "+f"(v[29]), "+f"(v[30]), "+f"(v[31])
               :
               : "memory");
}
// The wait for K (a multiple of 16) float32 registers filled by tmem_ld16, tied 32 at a
// time where K allows (with 16-register waits only, the 32^2 plane kernel spilled 8 bytes).
template <int K>
__device__ __forceinline__ void tmem_wait_ld(float* v) {
  static_assert(K % 16 == 0, "whole 16-column loads");
  if constexpr (K % 32 == 0) {
#pragma unroll
    for (int c = 0; c < K; c += 32) tmem_wait_ld32(v + c);
  } else {
#pragma unroll
    for (int c = 0; c < K; c += 16) tmem_wait_ld16(v + c);
  }
}

// N values of a pencil <-> consecutive TMEM columns of this thread's lane: float32 one
// column each, float64 two (low word, then high word).  The float32 load is completed by
// the caller's tmem_wait_pencil; the float64 load waits after each 16 columns and then
// assembles its 8 values, so no word is read before it has arrived.
template <typename T, int N>
__device__ __forceinline__ void tmem_st_pencil(uint32_t addr, const T* v) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int c = 0; c < N; c += 16) tmem_st16(addr + c, reinterpret_cast<const float*>(v) + c);
  } else {
#pragma unroll
    for (int c = 0; c < N; c += 8) {
      float w[16];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        w[2 * k] = __int_as_float(__double2loint((double)v[c + k]));
        w[2 * k + 1] = __int_as_float(__double2hiint((double)v[c + k]));
      }
      tmem_st16(addr + 2 * c, w);
    }
  }
}
template <typename T, int N>
__device__ __forceinline__ void tmem_ld_pencil(uint32_t addr, T* v) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int c = 0; c < N; c += 16) tmem_ld16(addr + c, reinterpret_cast<float*>(v) + c);
  } else {
#pragma unroll
    for (int c = 0; c < N; c += 8) {
      float w[16];
      tmem_ld16(addr + 2 * c, w);
      tmem_wait_ld16(w);
#pragma unroll
      for (int k = 0; k < 8; ++k) v[c + k] = (T)__hiloint2double(__float_as_int(w[2 * k + 1]), __float_as_int(w[2 * k]));
    }
  }
}
// Completes tmem_ld_pencil of a real and an imaginary pencil (float32: the tied wait;
// float64 pencils have been assembled after their own waits).
template <typename T, int N>
__device__ __forceinline__ void tmem_wait_pencil(T* re, T* im) {
  if constexpr (sizeof(T) == 4) {
    tmem_wait_ld<N>(reinterpret_cast<float*>(re));
    tmem_wait_ld<N>(reinterpret_cast<float*>(im));
  }
}

// ---- tensor-core 1D DFT of 128 pencils (tcgen05) ------------------------------------
// Each thread of the CTA holds one pencil of N complex values.  The inverse DFT of all
// 128 pencils is one dense contraction D[128 x 2N] = A[128 x 2N] W[2N x 2N] with the real
// block form A = [re | im], W = [[C, S], [-S, C]] (C, S = cos, sin of 2 pi x k / N): rows
// go to shared memory, one thread issues the MMAs (accumulator in TMEM), the others wait
// on an mbarrier with a bounded number of tries, and every thread reads its row back
// with tcgen05.ld.  Modes: TF32 (kind::tf32, operands rounded to tf32); 3xTF32 and
// 3xBF16 split both operands into high and low parts of that type and accumulate
// Ah Wh + Ah Wl + Al Wh (kind::tf32, or kind::f16 with bf16 operands); the Al Wl term is
// below the split's resolution.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// bf16 round-to-nearest-even of x, returned as its 16-bit pattern and its float value
__device__ __forceinline__ uint16_t to_bf16(float x, float& back) {
  uint16_t h;
  asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(x));
  back = __uint_as_float((uint32_t)h << 16);
  return h;
}

// shared-memory matrix descriptor: start, leading (K) and stride (8-row) byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

template <int N, int TC>
struct TcDft {
  static constexpr int K = 2 * N;
  static constexpr bool kBF16 = (TC == kTc3xBF16);
  static constexpr bool kSplit = (TC == kTc3xTF32 || TC == kTc3xBF16);
  static constexpr int ES = kBF16 ? 2 : 4;   // element bytes
  static constexpr int EPC = 16 / ES;        // elements per 16-byte core-matrix row
  static constexpr int SBO = (K / EPC) * 128;  // bytes between 8-row groups
  static constexpr int KSTEP = 32 / ES;      // K per MMA instruction (32 bytes)
  unsigned char* A;         // [split][128 x K] K-major, no swizzle
  const unsigned char* W;   // [split][K x K] as B operand rows n (output), K-major
  uint64_t* mbar;
  uint32_t tmem;
  uint32_t phase;

  // byte offset of element (row, k): 8-row x 16-byte core matrices, K-adjacent ones 128
  // bytes apart, 8-row groups SBO apart
  __device__ static __forceinline__ int offs(int row, int k) {
    return (row / 8) * SBO + (k / EPC) * 128 + (row % 8) * 16 + (k % EPC) * ES;
  }

  // the inverse-DFT matrix from the twiddle table, high (and low) parts
  __device__ static void build_w(unsigned char* Wdst, int t, int nthreads) {
    constexpr int stride = kTw / N;
    for (int i = t; i < K * K; i += nthreads) {
      const int nn = i / K, k = i % K;  // output index, input index
      const int x = nn % N, kk = k % N;
      const int m = (x * kk) % N;
      const float c = tw_cos<float>(m * stride), sn = tw_sin<float>(m * stride);
      float v;
      if (nn < N) v = (k < N) ? c : -sn;   // Re y = C Re a - S Im a
      else v = (k < N) ? sn : c;           // Im y = S Re a + C Im a
      if constexpr (kBF16) {
        float hb, lb;
        const uint16_t h = to_bf16(v, hb);
        const uint16_t l = to_bf16(v - hb, lb);
        *reinterpret_cast<uint16_t*>(Wdst + offs(nn, k)) = h;
        *reinterpret_cast<uint16_t*>(Wdst + K * K * ES + offs(nn, k)) = l;
      } else {
        const float hi = to_tf32(v);
        *reinterpret_cast<float*>(Wdst + offs(nn, k)) = hi;
        if constexpr (kSplit) *reinterpret_cast<float*>(Wdst + K * K * ES + offs(nn, k)) = to_tf32(v - hi);
      }
    }
  }

  __device__ __forceinline__ void mma_set(uint32_t a_addr, uint32_t b_addr, bool first) const {
    // D f32; A and B tf32 (2) or bf16 (1); both K-major; N = K; M = 128
    constexpr uint32_t fmt = kBF16 ? 1u : 2u;
    constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(K >> 3) << 17) | ((128u >> 4) << 24);
#pragma unroll
    for (int s = 0; s < K / KSTEP; ++s) {
      const uint64_t ad = umma_desc(a_addr + s * 256, 128, SBO);
      const uint64_t bd = umma_desc(b_addr + s * 256, 128, SBO);
      const uint32_t acc = (first && s == 0) ? 0u : 1u;
      if constexpr (kBF16) {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      } else {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
    }
  }

  // 8 values of the row (bf16: one 16-byte chunk; tf32: two) at k0, high and low parts
  __device__ __forceinline__ void put8(int t, int k0, const float* v) {
    if constexpr (kBF16) {
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float h0, h1, l0, l1;
        const uint16_t a0 = to_bf16(v[2 * q], h0), a1 = to_bf16(v[2 * q + 1], h1);
        const uint16_t b0 = to_bf16(v[2 * q] - h0, l0), b1 = to_bf16(v[2 * q + 1] - h1, l1);
        hw[q] = (uint32_t)a0 | ((uint32_t)a1 << 16);
        lw[q] = (uint32_t)b0 | ((uint32_t)b1 << 16);
      }
      *reinterpret_cast<uint4*>(A + offs(t, k0)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4*>(A + 128 * K * ES + offs(t, k0)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    } else {
#pragma unroll
      for (int q = 0; q < 8; q += 4) {
        const float4 h = make_float4(to_tf32(v[q]), to_tf32(v[q + 1]), to_tf32(v[q + 2]), to_tf32(v[q + 3]));
        *reinterpret_cast<float4*>(A + offs(t, k0 + q)) = h;
        if constexpr (kSplit)
          *reinterpret_cast<float4*>(A + 128 * K * ES + offs(t, k0 + q)) =
              make_float4(to_tf32(v[q] - h.x), to_tf32(v[q + 1] - h.y), to_tf32(v[q + 2] - h.z),
                          to_tf32(v[q + 3] - h.w));
      }
    }
  }

  // inverse DFT of this thread's pencil (re, im) in place; all 128 threads call it
  __device__ __forceinline__ void inverse(float (&re)[N], float (&im)[N], int t) {
#pragma unroll
    for (int k = 0; k < N; k += 8) {
      put8(t, k, re + k);
      put8(t, N + k, im + k);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (t == 0) {
      const uint32_t a0 = smem_u32(A), w0 = smem_u32(W);
      mma_set(a0, w0, true);
      if constexpr (kSplit) {
        mma_set(a0, w0 + K * K * ES, false);        // Ah Wl
        mma_set(a0 + 128 * K * ES, w0, false);      // Al Wh
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(mbar))
                   : "memory");
    }
    uint32_t done = 0;
    for (int it = 0; it < (1 << 20) && !done; ++it) {
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(smem_u32(mbar)), "r"(phase)
          : "memory");
    }
    if (!done) atomicOr(&g_boltz_status, kStatusTimeout);
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t lane_base = tmem + ((uint32_t)((t >> 5) * 32) << 16);
#pragma unroll
    for (int c = 0; c < K; c += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(lane_base + c));
      tmem_wait_ld16(r);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = c + j;
        if (col < N) re[col] = __uint_as_float(r[j]);
        else im[col - N] = __uint_as_float(r[j]);
      }
    }
  }
};

template <typename T, typename TIO, int N, int C, bool kSplit, int TC = kTcNone>
__global__ void __launch_bounds__(CollideCfg<T, N, C, TC>::THREADS, CollideCfg<T, N, C, TC>::MIN_BLOCKS)
collide_kernel(const CollideArgs args) {
  using Cfg = CollideCfg<T, N, C, TC>;
  static_assert(!(kSplit && TC != kTcNone), "tensor-core transforms run without term groups");
  using T2 = typename Cfg::T2;
  constexpr int NP = Cfg::NP, WARPS = Cfg::WARPS, VEC = Cfg::VEC, NCH = Cfg::NCH, RW_ = Cfg::RW;
  constexpr int n = N * N * N;
  constexpr bool kRegSpec = Cfg::kRegSpec;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  T2* Fh = reinterpret_cast<T2*>(smem_raw);                       // unused when kRegSpec
  T2* XB0 = reinterpret_cast<T2*>(smem_raw + Cfg::OFF_XB);
  double* red = reinterpret_cast<double*>(smem_raw + Cfg::OFF_RED);

  const int rank = (C > 1) ? (int)cg::this_cluster().block_rank() : 0;
  // Cell of the launch and term group of this cluster.
  const int G = kSplit ? args.groups : 1;
  long long lc = blockIdx.x / C;
  int gi = 0;
  if constexpr (kSplit) {
    gi = (int)(lc % G);
    lc /= G;
  }
  // Slot of this cell.  An index outside [0, pool_cells) is reported; the cell then
  // reads slot 0 and writes nothing, so every CTA still runs the same barrier sequence.
  long long cell = lc;
  bool writable = true;
  if (args.cell_idx) {
    const long long s = args.cell_idx[cell];
    writable = (s >= 0 && s < args.pool_cells);
    if (!writable && threadIdx.x == 0) atomicOr(&g_boltz_status, kStatusBadIndex);
    cell = writable ? s : 0;
  }
  const int t = threadIdx.x;
  // spectral passes: thread (kyl, kz), lanes along kz
  const int kyl = t / N, kzt = t % N;
  // physical passes: thread (xl, ky) in the kz pass, (xl, z) in the ky pass / epilogue,
  // lanes ordered (xl % VEC, ky or z), xl / VEC slowest
  const int xlt = (t / (VEC * N)) * VEC + t % VEC, grp = (t / VEC) % N;
  const int zt = grp;
  const T2* tab = reinterpret_cast<const T2*>(args.tab);
  const int M_eff = args.M_eff;
  const int ky_own = rank * NP + kyl;  // spectral ky of this thread's pencils
  const int x_own = rank * NP + xlt;   // physical x of this thread's rows
  const TIO* fin = cell_input<TIO>(args, cell, x_own, n);

  T re[N], im[N];
  constexpr bool kTmemSpec = Cfg::kTmemSpec;
  constexpr bool kRegArr = kRegSpec && !kTmemSpec;
  T fr[kRegArr ? N : 1], fi[kRegArr ? N : 1];  // spectrum pencil in registers (tensor-core modes)
  uint32_t spec_re = 0, spec_im = 0;  // spectrum pencil in TMEM: real and imaginary halves
  uint32_t* spec_slots = reinterpret_cast<uint32_t*>(smem_raw + Cfg::OFF_TSLOT);
  if constexpr (kTmemSpec) {
    // one allocation of TMEM_COLS, or one kTmemShare-column share per group of four warps
    if ((threadIdx.x >> 5) == 0) {
#pragma unroll
      for (int k = 0; k < Cfg::TMEM_SHARES; ++k)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(spec_slots + k)),
                     "r"(Cfg::TMEM_SHARES == 1 ? Cfg::TMEM_COLS : kTmemShare));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int grp4 = threadIdx.x >> 7;  // group of four warps: lanes 0..127 of a column group
    const uint32_t lane_off = (uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16;
    if constexpr (Cfg::TMEM_SHARES == 1) {
      spec_re = spec_slots[0] + (uint32_t)(grp4 * Cfg::GROUP_COLS) + lane_off;
      spec_im = spec_re + (uint32_t)(N * Cfg::CPV);
    } else if constexpr (Cfg::SPG == 1) {
      spec_re = spec_slots[grp4] + lane_off;
      spec_im = spec_re + (uint32_t)(N * Cfg::CPV);
    } else {
      spec_re = spec_slots[2 * grp4] + lane_off;
      spec_im = spec_slots[2 * grp4 + 1] + lane_off;
    }
  }

  // tensor-core transforms: TMEM accumulator (2N columns), completion barrier, DFT matrix
  TcDft<N, TC> tc;
  if constexpr (TC != kTcNone) {
    tc.A = smem_raw + Cfg::OFF_TCA;
    tc.W = smem_raw + Cfg::OFF_TCW;
    tc.mbar = reinterpret_cast<uint64_t*>(smem_raw + Cfg::OFF_TCB);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem_raw + Cfg::OFF_TCB + 8);
    if ((threadIdx.x >> 5) == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(Cfg::TC_TMEM_COLS));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(tc.mbar)));
      asm volatile("fence.mbarrier_init.release.cluster;");
    }
    TcDft<N, TC>::build_w(smem_raw + Cfg::OFF_TCW, threadIdx.x, Cfg::THREADS);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tc.tmem = *tmem_slot;
    tc.phase = 0u;
  }
  // asynchronous scatter (32^3 single-buffer layout): the owner has one mbarrier per
  // chunk of its x-slab (chunk c: the x-planes c VEC .. c VEC + VEC - 1, whose kz and ky
  // passes are done by threads [c THREADS / NCH, (c + 1) THREADS / NCH) alone), counting
  // the bytes that reach that chunk of its buffer, so the warps of a chunk start as soon
  // as their planes have landed.  Each is armed for term 0 at initialisation (before this
  // CTA's first write-after-read arrive) and re-armed for term i + 1 by the chunk's first
  // thread right after its wait for term i (before the arrive of term i), so no bytes of
  // a term can arrive before their phase is armed
  constexpr bool kAsync = Cfg::kAsyncScatter;
  const uint32_t scat_mbar = smem_u32(smem_raw + Cfg::OFF_MBAR);
  uint32_t scat_phase = 0;
  if constexpr (kAsync) {
    if (threadIdx.x == 0) {
      for (int c = 0; c < Cfg::NCH; ++c) mbar_init(scat_mbar + 8 * c, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      // term 0's phases, armed before any arrive
      for (int c = 0; c < Cfg::NCH; ++c) mbar_expect_tx(scat_mbar + 8 * c, Cfg::SCATTER_BYTES / Cfg::NCH);
    }
  }
  // inverse 1D transform of this thread's pencil: register FFT or tensor-core DFT
  auto inverse_1d = [&]() {
    if constexpr (TC != kTcNone) {
      tc.inverse(re, im, threadIdx.x);
    } else {
      fft_regs<N, +1>(re, im);
    }
  };

  const double L = args.geom.L, dv = args.geom.dv;
  const int lane = t & 31, warp = t >> 5;
  // ---- forward transform, pass along y: thread (x, z) --------------------------------
  {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;  // sum_y f, sum_y y f, sum_y y^2 f (targets)
#pragma unroll
    for (int y = 0; y < N; ++y) {
      const TIO fv = fin[(x_own * N + y) * N + zt];
      re[y] = (T)fv;
      im[y] = T(0);
      if (args.compute_targets) {
        s0 += (double)fv;
        s1 += (double)y * (double)fv;
        s2 += (double)(y * y) * (double)fv;
      }
    }
    if (args.compute_targets) {
      // Phi f over this thread's y-row: v_y = -L + y dv
      const double vx = -L + x_own * dv, vz = -L + zt * dv;
      const double sy = -L * s0 + dv * s1;                              // sum v_y f
      const double syy = L * L * s0 - 2.0 * L * dv * s1 + dv * dv * s2;  // sum v_y^2 f
      double m[5] = {s0, vx * s0, sy, vz * s0, 0.5 * ((vx * vx + vz * vz) * s0 + syy)};
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        const double v = warp_sum(m[r]);
        if (lane == 0) red[warp * 5 + r] = v;
      }
    }
    fft_regs<N, -1>(re, im);
#pragma unroll
    for (int k = 0; k < N; ++k) XB0[Cfg::elem(xlt, k, zt)] = mk2<T>(re[k], im[k]);
  }
  __syncthreads();
  if (args.compute_targets && t < 5) {
    double v = 0.0;
    for (int w = 0; w < WARPS; ++w) v += red[w * 5 + t];
    red[(WARPS + 1) * 5 + t] = v;  // this CTA's Phi f_in
  }
  // ---- pass along z: thread (xl, ky) ----------------------------------------------------
  {
    T2* col = XB0 + Cfg::elem(xlt, grp, 0);
#pragma unroll
    for (int z = 0; z < N; ++z) {
      const T2 v = col[z * VEC];
      re[z] = v.x;
      im[z] = v.y;
    }
    fft_regs<N, -1>(re, im);
#pragma unroll
    for (int k = 0; k < N; ++k) col[k * VEC] = mk2<T>(re[k], im[k]);
  }
  cluster_barrier<C>();
  // ---- pass along x, gathering the peers' x-planes: thread (kyl, kz) -------------------
  {
    // chunk c of CTA q holds x = q NP + c VEC + (0 .. VEC-1)
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      const T2* src = XB0 + Cfg::elem(c * VEC, ky_own, kzt);
      if constexpr (C > 1) {
        const uint32_t a = smem_u32(src);
#pragma unroll
        for (int q = 0; q < C; ++q) ld_cluster_chunk(cluster_addr(a, q), re + q * NP + c * VEC, im + q * NP + c * VEC);
      } else {
        ld_local_chunk(src, re + c * VEC, im + c * VEC);
      }
    }
    // Single buffer: the peers must be done gathering from this CTA's x-planes before
    // the first scatter into them.  In a cluster the barrier is split: this arrive, right
    // after the last gather (a release: it orders the gathers before the peers' stores),
    // and the wait inside the first kx pass just before its stores.
    if constexpr (Cfg::NXB == 1 && C > 1) cluster_arrive_war<C>();
    fft_regs<N, -1>(re, im);
    const T scale = T(1) / T(n);
    const bool nyq = (ky_own == N / 2) || (kzt == N / 2);
#pragma unroll
    for (int kx = 0; kx < N; ++kx) {
      // Every mode with a component -N/2 is removed so each inverse transform is real.
      const bool z0 = nyq || (kx == N / 2);
      const T vr = z0 ? T(0) : re[kx] * scale, vi = z0 ? T(0) : im[kx] * scale;
      if constexpr (kTmemSpec) {
        re[kx] = vr;
        im[kx] = vi;
      } else if constexpr (kRegSpec) {
        fr[kx] = vr;
        fi[kx] = vi;
      } else {
        Fh[(kx * NP + kyl) * N + kzt] = mk2<T>(vr, vi);
      }
    }
    if constexpr (kTmemSpec) {
      tmem_st_pencil<T, N>(spec_re, re);
      tmem_st_pencil<T, N>(spec_im, im);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
  }
  // Single buffer without a cluster: the CTA's own gathers end before its first scatter.
  constexpr bool kSplitWar = (Cfg::NXB == 1) && (C > 1);
  if constexpr (Cfg::NXB == 1 && C == 1) __syncthreads();

  // ---- angular loop: one complex inverse transform per separated term --------------
  T acc[N];
#pragma unroll
  for (int y = 0; y < N; ++y) acc[y] = T(0);

  // pass along kx with the coefficients of term j: thread (kyl, kz), tables from L2;
  // outputs x = q NP + c VEC + (0 .. VEC-1) go to chunk c of CTA q at (ky, kz)
  auto pass_kx = [&](int j, T2* XB) {
    const T2* tj = tab + (size_t)j * n + (size_t)ky_own * N * N + kzt;
    if constexpr (kTmemSpec) {
      tmem_ld_pencil<T, N>(spec_re, re);
      tmem_ld_pencil<T, N>(spec_im, im);
      tmem_wait_pencil<T, N>(re, im);
    }
#pragma unroll
    for (int kx = 0; kx < N; ++kx) {
      T2 c;
      if constexpr (kTmemSpec) {
        c = mk2<T>(re[kx], im[kx]);
      } else if constexpr (kRegSpec) {
        c = mk2<T>(fr[kx], fi[kx]);
      } else {
        c = Fh[(kx * NP + kyl) * N + kzt];
      }
      const T2 ab = __ldg(tj + kx * N);
      re[kx] = ab.x * c.x - ab.y * c.y;
      im[kx] = ab.x * c.y + ab.y * c.x;
    }
    inverse_1d();
    if constexpr (kSplitWar) cluster_wait_war<C>();  // every owner has read its buffer
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      T2* dst = XB + Cfg::elem(c * VEC, ky_own, kzt);
      if constexpr (kAsync) {
        const uint32_t a = smem_u32(dst);
#pragma unroll
        for (int q = 0; q < C; ++q)
          st_async_chunk(cluster_addr(a, q), reinterpret_cast<const float*>(re) + q * NP + c * VEC,
                         reinterpret_cast<const float*>(im) + q * NP + c * VEC, cluster_addr(scat_mbar + 8 * c, q));
      } else if constexpr (C > 1) {
        const uint32_t a = smem_u32(dst);
#pragma unroll
        for (int q = 0; q < C; ++q) st_cluster_chunk(cluster_addr(a, q), re + q * NP + c * VEC, im + q * NP + c * VEC);
      } else {
        st_local_chunk(dst, re + c * VEC, im + c * VEC);
      }
    }
  };
  // pass along kz: thread (xl, ky)
  auto pass_kz = [&](T2* XB) {
    T2* col = XB + Cfg::elem(xlt, grp, 0);
#pragma unroll
    for (int kz = 0; kz < N; ++kz) {
      const T2 v = col[kz * VEC];
      re[kz] = v.x;
      im[kz] = v.y;
    }
    inverse_1d();
#pragma unroll
    for (int z = 0; z < N; ++z) col[z * VEC] = mk2<T>(re[z], im[z]);
  };
  // pass along ky: thread (xl, z); outputs along y.  accumulate: Q+ += w Re Im; otherwise
  // re[] keeps the loss multiplier L(v) along y.  release: these loads were this CTA's
  // last reads of its x-plane buffer for the term, so the write-after-read arrive (a
  // release, which orders them before the peers' next stores) ends the pass.  (Placed
  // right after the loads instead, it measured slower: the release then also waits for
  // the loads and for the term's scatter stores still in flight.)
  auto pass_ky = [&](const T2* XB, T wj, bool accumulate, bool release) {
    const T2* col = XB + Cfg::elem(xlt, 0, zt);
#pragma unroll
    for (int ky = 0; ky < N; ++ky) {
      const T2 v = col[ky * (RW_ * VEC)];
      re[ky] = v.x;
      im[ky] = v.y;
    }
    inverse_1d();
    if (accumulate) {
#pragma unroll
      for (int y = 0; y < N; ++y) acc[y] += wj * (re[y] * im[y]);
    }
    if constexpr (Cfg::NXB == 1 && C > 1) {
      if (release) {
        if constexpr (kAsync) {
          // the chunk's threads meet (its named barrier, which orders their loads before
          // what its threads do next); the chunk's first warp then arrives with .release,
          // cumulative over all those loads, and the other warps relaxed: one warp per
          // chunk pays for the release instead of every thread
          asm volatile("bar.sync %0, %1;" ::"r"(1 + xlt / VEC), "r"(Cfg::THREADS / Cfg::NCH) : "memory");
          if (((threadIdx.x % (Cfg::THREADS / Cfg::NCH)) >> 5) == 0) {
            cluster_arrive_war<C>();
          } else {
            asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
          }
        } else {
          cluster_arrive_war<C>();
        }
      }
    }
  };

  // This cluster's terms: i = 0 .. nt-1 is term j0 + i, and the loss transform (term
  // M_eff) comes last in the last group (without a split: i = j = 0 .. M_eff).
  const int j0 = kSplit ? (int)(((long long)gi * M_eff) / G) : 0;
  const int j1 = kSplit ? (int)(((long long)(gi + 1) * M_eff) / G) : M_eff;
  const bool has_loss = kSplit ? (gi == G - 1) : true;
  const int nt = (j1 - j0) + (has_loss ? 1 : 0);
  if constexpr (Cfg::NXB == 2) {
    // Two x-plane buffers; term i uses buffer (i + 1) % 2.  The ky pass of term i - 1
    // runs between the scatter of term i and the cluster barrier, so the remote stores
    // drain behind it.  It reads the other buffer, and every CTA finishes it before
    // arriving, so no peer scatters term i + 1 into that buffer while it is read.
    T w_prev = T(0);
    for (int i = 0; i < nt; ++i) {
      const int j = kSplit ? ((j0 + i < j1) ? j0 + i : M_eff) : i;
      T2* XBj = XB0 + ((i + 1) & 1) * Cfg::XB;
      const T wj = (j < M_eff) ? (T)args.w[j] : T(0);
      pass_kx(j, XBj);
      if (i > 0) pass_ky(XB0 + (i & 1) * Cfg::XB, w_prev, true, false);
      cluster_barrier<C>();
      pass_kz(XBj);
      __syncthreads();
      w_prev = wj;
    }
    // last term: the loss transform (re[] keeps L) or a gain term
    if (has_loss) {
      pass_ky(XB0 + (nt & 1) * Cfg::XB, T(0), false, false);
    } else {
      pass_ky(XB0 + (nt & 1) * Cfg::XB, w_prev, true, false);
    }
  } else {
    for (int i = 0; i < nt; ++i) {
      const int j = kSplit ? ((j0 + i < j1) ? j0 + i : M_eff) : i;
      const T wj = (j < M_eff) ? (T)args.w[j] : T(0);
      pass_kx(j, XB0);
      const bool more = (i < nt - 1);
      if constexpr (kAsync) {
        // every producer's bytes of this term have landed in this thread's chunk
        const uint32_t my_mbar = scat_mbar + 8 * (xlt / VEC);
        if (!mbar_wait(my_mbar, scat_phase)) atomicOr(&g_boltz_status, kStatusTimeout);
        scat_phase ^= 1u;
        // arm the chunk's next phase now: its bytes cannot come before this CTA's
        // write-after-read arrive below
        if (more && (threadIdx.x % (Cfg::THREADS / Cfg::NCH)) == 0) mbar_expect_tx(my_mbar, Cfg::SCATTER_BYTES / Cfg::NCH);
      } else {
        cluster_barrier<C>();
      }
      pass_kz(XB0);
      if constexpr (kAsync) {
        // the chunk's own threads wrote its planes: a barrier among them (ids 1 ..)
        asm volatile("bar.sync %0, %1;" ::"r"(1 + xlt / VEC), "r"(Cfg::THREADS / Cfg::NCH) : "memory");
      } else {
        __syncthreads();
      }
      // single buffer: the owners' last reads of term i (the ky loads) come before the
      // arrive (end of pass_ky) that lets the peers scatter term i + 1 (their wait is in
      // pass_kx)
      pass_ky(XB0, wj, j < M_eff, more && kSplitWar);
      if constexpr (!kSplitWar) {
        if (more) cluster_barrier_war<C>();
      }
    }
    if constexpr (kSplitWar) {
      if (nt == 0) cluster_wait_war<C>();  // a group without terms: close the first arrive
    }
  }

  if constexpr (kTmemSpec) {
    // the spectrum is no longer needed: free its TMEM columns
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
#pragma unroll
      for (int k = 0; k < Cfg::TMEM_SHARES; ++k)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(spec_slots[k]),
                     "r"(Cfg::TMEM_SHARES == 1 ? Cfg::TMEM_COLS : kTmemShare));
    }
  }
  if constexpr (TC != kTcNone) {
    // every thread has read its last accumulator row: free the TMEM columns
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc.tmem), "r"(Cfg::TC_TMEM_COLS));
  }
  if constexpr (kSplit) {
    // Partial gain (and the loss multiplier) of this group, then the last-arrival count
    // of the cell (fence, barrier, one atomic: no waiting).  The cluster that arrives last
    // sums the G partials in group order, so the result does not depend on the order of
    // arrival, and continues with the epilogue; the others leave.
    T* part;
    T* lossp;
    unsigned* arrp;
    split_scratch<T>(args, lc, G, n, part, lossp, arrp);
#pragma unroll
    for (int y = 0; y < N; ++y) {
      const int idx = (x_own * N + y) * N + zt;
      part[(size_t)gi * n + idx] = acc[y];
      if (has_loss) lossp[idx] = re[y];
    }
    __threadfence();
    cluster_barrier<C>();
    unsigned* flag = reinterpret_cast<unsigned*>(smem_raw + Cfg::OFF_FLAG);
    if (rank == 0 && t == 0) {
      const unsigned prev = atomicAdd(arrp, 1u);
      const unsigned last = (prev == (unsigned)(G - 1)) ? 1u : 0u;
      if (last) *arrp = 0u;  // every group has arrived: ready for the next launch
#pragma unroll
      for (int q = 0; q < C; ++q) *cta_smem<C>(flag, q) = last;
    }
    cluster_barrier<C>();
    if (*flag == 0u) return;  // the whole cluster leaves together
    __threadfence();
#pragma unroll
    for (int y = 0; y < N; ++y) {
      const int idx = (x_own * N + y) * N + zt;
      T sum = __ldcg(part + idx);
      for (int g2 = 1; g2 < G; ++g2) sum += __ldcg(part + (size_t)g2 * n + idx);
      acc[y] = sum;
      re[y] = __ldcg(lossp + idx);
    }
  }

  // ---- Q = Q+ - f L, projection and update (float64): thread (x, z) ------------------
  const int x = x_own, z = zt;
  const double vx = -L + x * dv, vz = -L + z * dv;
  const TIO* fb = args.f_base ? reinterpret_cast<const TIO*>(args.f_base) + cell * n : nullptr;
  double g[N];
  double S0 = 0.0, S1 = 0.0, S2 = 0.0;  // sum_y g, sum_y y g, sum_y y^2 g over this row
#pragma unroll
  for (int y = 0; y < N; ++y) {
    const int idx = (x * N + y) * N + z;
    const TIO fv = fin[idx];
    const T q = acc[y] - (T)fv * re[y];  // Q = Q+ - f L (one rounding in T)
    double gv = args.s * (double)q;
    if (args.b != 0.0) gv += args.b * (double)fv;
    if (fb) gv += args.a * (double)fb[idx];
    g[y] = gv;
    S0 += gv;
    S1 += (double)y * gv;
    S2 += (double)(y * y) * gv;
  }
  // Phi g over the row, with v_y = -L + y dv
  double m[5] = {S0, vx * S0, -L * S0 + dv * S1, vz * S0,
                 0.5 * ((vx * vx + vz * vz + L * L) * S0 - 2.0 * L * dv * S1 + dv * dv * S2)};
  double c5[5];
  cluster_correction<C, WARPS>(args, m, red, cell, writable, rank, t, c5);
  TIO* out = reinterpret_cast<TIO*>(args.out) + cell * n;
  bool bad = false;
  // Phi^T c at (vx, vy, vz) as a quadratic in the row index y: P0 + P1 y + P2 y^2
  const double P0 = c5[0] + c5[1] * vx + c5[3] * vz + 0.5 * c5[4] * (vx * vx + vz * vz + L * L) - c5[2] * L;
  const double P1 = (c5[2] - c5[4] * L) * dv;
  const double P2 = 0.5 * c5[4] * dv * dv;
#pragma unroll
  for (int y = 0; y < N; ++y) {
    const double val = g[y] + (P0 + (double)y * (P1 + (double)y * P2));
    bad |= !isfinite(val);
    if (writable) out[(x * N + y) * N + z] = (TIO)val;
  }
  if (bad) atomicOr(&g_boltz_status, kStatusNonFinite);
}

// ------------------------------------------------------------------------------------
// N = 48 and 64 (float32).  One pencil of 48 or 64 complex values takes 96 or 128
// registers, so the gain accumulator and the spectrum cannot stay in registers as above:
// each thread's spectrum pencil goes to tensor memory (written once, read back by the
// same thread every term, in 64-column shares), the gain accumulator of the CTA's
// x-slab lives in shared memory, and one x-plane buffer serves every term with the
// 32^3 kernel's exchange (st.async scatter, per-chunk waits, split write-after-read
// barrier).  Clusters of 12 at 48^3 (4 x-planes per CTA, two CTAs per SM) and of 16 at
// 64^3 (one CTA per SM).  The epilogue recomputes g in a second sweep instead of
// keeping N float64 values per thread.  Otherwise the same decomposition and arithmetic
// as collide_kernel.
// ------------------------------------------------------------------------------------
template <int N, int C>
struct LargeCfg {
  static constexpr int NP = N / C;
  static constexpr int THREADS = NP * N;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int VEC = 2;
  static constexpr int NCH = NP / VEC;
  static constexpr int RW = N + 1;
  static constexpr size_t XB = (size_t)NCH * N * RW * VEC;        // float2
  // gain accumulator [xl][y][z], float; consecutive x-planes ACC_PLANE floats apart, with
  // ACC_PLANE = 16 (mod 32) so that the two x-values of a warp (lanes ordered (x % 2, z))
  // fall in opposite halves of the 32 banks (an N^2 stride, 0 mod 32, put them in one)
  static constexpr int ACC_PLANE = N * N + ((16 - (N * N) % 32) + 32) % 32;
  static constexpr size_t ACC = (size_t)NP * ACC_PLANE;
  static constexpr size_t OFF_ACC = XB * sizeof(float2);
  static constexpr size_t OFF_RED = OFF_ACC + ACC * sizeof(float);
  static constexpr size_t OFF_FLAG = OFF_RED + (size_t)(WARPS + 2) * 5 * sizeof(double);
  // flag, then one scatter mbarrier per chunk of the x-slab, then the TMEM addresses
  static constexpr size_t OFF_MBAR = OFF_FLAG + 16;
  // spectrum pencils in TMEM: warp w uses lanes 32 (w % 4) .. + 31; each group of four
  // warps holds two kTmemShare-column allocations, its N real parts in one and its N
  // imaginary parts in the other, so the kernel follows the share rule above
  static constexpr int GROUPS4 = (WARPS + 3) / 4;
  static constexpr int TMEM_SHARES = 2 * GROUPS4;
  static constexpr size_t OFF_TSLOT = OFF_MBAR + 8 * NCH;
  static constexpr size_t SMEM = (OFF_TSLOT + 4 * TMEM_SHARES + 15) / 16 * 16;
  // CTAs per SM: two at 48^3 with 12-CTA clusters (4 x-planes, 192 threads, 110 KB of
  // shared memory, 4 shares), one otherwise
  static constexpr int MIN_BLOCKS = (N == 48 && C == 12) ? 2 : 1;
  // bytes a CTA receives per term (its x-slab of one term's kx-pass outputs)
  static constexpr uint32_t SCATTER_BYTES = (uint32_t)NP * N * N * 2 * sizeof(float);
  static_assert(NCH <= 4 && (THREADS / NCH) % 32 == 0, "per-chunk mbarriers and named barriers");
  static_assert(N <= kTmemShare && TMEM_SHARES <= 8, "real or imaginary parts of a pencil fit one share");
  static_assert(N % 16 == 0, "whole 16-column TMEM chunks");
  static_assert(THREADS % 32 == 0 && NP % VEC == 0, "whole warps and chunks");
  static_assert(OFF_RED % 16 == 0, "aligned reduction area");
  static_assert(ACC_PLANE % 32 == 16 && ACC_PLANE >= N * N, "x-planes of the accumulator in opposite bank halves");
  static_assert(SMEM <= 232448, "shared memory per CTA");
  static __device__ __forceinline__ int elem(int xl, int ky, int k) {
    return ((xl / VEC) * N + ky) * RW * VEC + k * VEC + xl % VEC;
  }
};

template <typename TIO, int N, int C, bool kSplit>
__global__ void __launch_bounds__(LargeCfg<N, C>::THREADS, LargeCfg<N, C>::MIN_BLOCKS)
    collide_large_kernel(const CollideArgs args) {
  using Cfg = LargeCfg<N, C>;
  using T = float;
  using T2 = float2;
  constexpr int NP = Cfg::NP, WARPS = Cfg::WARPS, VEC = Cfg::VEC, NCH = Cfg::NCH, RW_ = Cfg::RW;
  constexpr int n = N * N * N;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  T2* XB = reinterpret_cast<T2*>(smem_raw);
  float* accs = reinterpret_cast<float*>(smem_raw + Cfg::OFF_ACC);
  double* red = reinterpret_cast<double*>(smem_raw + Cfg::OFF_RED);

  const int rank = (C > 1) ? (int)cg::this_cluster().block_rank() : 0;
  const int G = kSplit ? args.groups : 1;
  long long lc = blockIdx.x / C;
  int gi = 0;
  if constexpr (kSplit) {
    gi = (int)(lc % G);
    lc /= G;
  }
  long long cell = lc;
  bool writable = true;
  if (args.cell_idx) {
    const long long s = args.cell_idx[cell];
    writable = (s >= 0 && s < args.pool_cells);
    if (!writable && threadIdx.x == 0) atomicOr(&g_boltz_status, kStatusBadIndex);
    cell = writable ? s : 0;
  }
  const int t = threadIdx.x;
  const int kyl = t / N, kzt = t % N;
  const int xlt = (t / (VEC * N)) * VEC + t % VEC, grp = (t / VEC) % N;
  const int zt = grp;
  const T2* tab = reinterpret_cast<const T2*>(args.tab);
  const int M_eff = args.M_eff;
  const int ky_own = rank * NP + kyl;
  const int x_own = rank * NP + xlt;
  const TIO* fin = cell_input<TIO>(args, cell, x_own, n);
  // this thread's spectrum pencil (its (ky, kz), all kx) in TMEM, written once by the
  // forward x pass and read back in every kx pass
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem_raw + Cfg::OFF_TSLOT);
  if ((t >> 5) == 0) {
#pragma unroll
    for (int k = 0; k < Cfg::TMEM_SHARES; ++k)
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot + k)),
                   "r"(kTmemShare));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t lane_off = (uint32_t)(32 * ((t >> 5) & 3)) << 16;
  const uint32_t spec_re = tmem_slot[2 * (t >> 7)] + lane_off, spec_im = tmem_slot[2 * (t >> 7) + 1] + lane_off;
  // Exchange per term as in collide_kernel's 32^3 single-buffer form: st.async scatter
  // completing on one mbarrier per chunk of the owner's x-slab (chunk c: planes c VEC ..,
  // whose kz and ky passes are done by threads [c THREADS / NCH, ...) alone), armed for
  // term 0 here, before this CTA's first write-after-read arrive, and re-armed by the
  // chunk's first thread right after its wait for each term.
  const uint32_t scat_mbar = smem_u32(smem_raw + Cfg::OFF_MBAR);
  uint32_t scat_phase = 0;
  if (t == 0) {
    for (int c = 0; c < NCH; ++c) mbar_init(scat_mbar + 8 * c, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int c = 0; c < NCH; ++c) mbar_expect_tx(scat_mbar + 8 * c, Cfg::SCATTER_BYTES / NCH);
  }
  const int chunk = xlt / VEC;  // this thread's chunk in the kz and ky passes
  constexpr int CH_THREADS = Cfg::THREADS / NCH;

  T re[N], im[N];
  const double L = args.geom.L, dv = args.geom.dv;
  const int lane = t & 31, warp = t >> 5;
  // ---- forward transform: y pass (thread (x, z)), z pass, x pass ----------------------
  {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int y = 0; y < N; ++y) {
      const TIO fv = fin[(x_own * N + y) * N + zt];
      re[y] = (T)fv;
      im[y] = T(0);
      if (args.compute_targets) {
        s0 += (double)fv;
        s1 += (double)y * (double)fv;
        s2 += (double)(y * y) * (double)fv;
      }
    }
    if (args.compute_targets) {
      const double vx = -L + x_own * dv, vz = -L + zt * dv;
      const double sy = -L * s0 + dv * s1;
      const double syy = L * L * s0 - 2.0 * L * dv * s1 + dv * dv * s2;
      double m[5] = {s0, vx * s0, sy, vz * s0, 0.5 * ((vx * vx + vz * vz) * s0 + syy)};
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        const double v = warp_sum(m[r]);
        if (lane == 0) red[warp * 5 + r] = v;
      }
    }
    fft_regs<N, -1>(re, im);
#pragma unroll
    for (int k = 0; k < N; ++k) XB[Cfg::elem(xlt, k, zt)] = make_float2(re[k], im[k]);
  }
  __syncthreads();
  if (args.compute_targets && t < 5) {
    double v = 0.0;
    for (int w = 0; w < WARPS; ++w) v += red[w * 5 + t];
    red[(WARPS + 1) * 5 + t] = v;
  }
  {
    T2* col = XB + Cfg::elem(xlt, grp, 0);
#pragma unroll
    for (int z = 0; z < N; ++z) {
      const T2 v = col[z * VEC];
      re[z] = v.x;
      im[z] = v.y;
    }
    fft_regs<N, -1>(re, im);
#pragma unroll
    for (int k = 0; k < N; ++k) col[k * VEC] = make_float2(re[k], im[k]);
  }
  cluster_barrier<C>();
  {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      const T2* src = XB + Cfg::elem(c * VEC, ky_own, kzt);
      const uint32_t a = smem_u32(src);
#pragma unroll
      for (int q = 0; q < C; ++q) ld_cluster_chunk(cluster_addr(a, q), re + q * NP + c * VEC, im + q * NP + c * VEC);
    }
    // the peers must be done gathering from this CTA's buffer before the first scatter
    // into it: this arrive (a release, ordering the gathers) and the wait in the first kx
    // pass, just before its stores
    cluster_arrive_war<C>();
    fft_regs<N, -1>(re, im);
    const T scale = T(1) / T(n);
    const bool nyq = (ky_own == N / 2) || (kzt == N / 2);
#pragma unroll
    for (int kx = 0; kx < N; ++kx) {
      const bool z0 = nyq || (kx == N / 2);
      re[kx] = z0 ? 0.f : re[kx] * scale;
      im[kx] = z0 ? 0.f : im[kx] * scale;
    }
#pragma unroll
    for (int c = 0; c < N; c += 16) {
      tmem_st16(spec_re + c, re + c);
      tmem_st16(spec_im + c, im + c);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  {  // this thread's row of the gain accumulator
    float* a = accs + (size_t)xlt * Cfg::ACC_PLANE + zt;
#pragma unroll
    for (int y = 0; y < N; ++y) a[y * N] = 0.f;
  }

  // ---- angular loop --------------------------------------------------------------------
  const int j0 = kSplit ? (int)(((long long)gi * M_eff) / G) : 0;
  const int j1 = kSplit ? (int)(((long long)(gi + 1) * M_eff) / G) : M_eff;
  const bool has_loss = kSplit ? (gi == G - 1) : true;
  const int nt = (j1 - j0) + (has_loss ? 1 : 0);
  for (int i = 0; i < nt; ++i) {
    const int j = kSplit ? ((j0 + i < j1) ? j0 + i : M_eff) : i;
    const T wj = (j < M_eff) ? (T)args.w[j] : T(0);
    {  // kx pass with the coefficients: thread (kyl, kz); outputs scattered by x
      const T2* tj = tab + (size_t)j * n + (size_t)ky_own * N * N + kzt;
#pragma unroll
      for (int c = 0; c < N; c += 16) {
        tmem_ld16(spec_re + c, re + c);
        tmem_ld16(spec_im + c, im + c);
      }
      tmem_wait_ld<N>(re);
      tmem_wait_ld<N>(im);
#pragma unroll
      for (int kx = 0; kx < N; ++kx) {
        const float cr = re[kx], cim = im[kx];
        const T2 ab = __ldg(tj + kx * N);
        re[kx] = ab.x * cr - ab.y * cim;
        im[kx] = ab.x * cim + ab.y * cr;
      }
      fft_regs<N, +1>(re, im);
      cluster_wait_war<C>();  // every owner has read its buffer
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        const uint32_t a = smem_u32(XB + Cfg::elem(c * VEC, ky_own, kzt));
#pragma unroll
        for (int q = 0; q < C; ++q)
          st_async_chunk(cluster_addr(a, q), re + q * NP + c * VEC, im + q * NP + c * VEC,
                         cluster_addr(scat_mbar + 8 * c, q));
      }
    }
    const bool more = (i < nt - 1);
    {  // every producer's bytes of this term have landed in this thread's chunk
      const uint32_t my_mbar = scat_mbar + 8 * chunk;
      if (!mbar_wait(my_mbar, scat_phase)) atomicOr(&g_boltz_status, kStatusTimeout);
      scat_phase ^= 1u;
      if (more && (t % CH_THREADS) == 0) mbar_expect_tx(my_mbar, Cfg::SCATTER_BYTES / NCH);
    }
    {  // kz pass: thread (xl, ky)
      T2* col = XB + Cfg::elem(xlt, grp, 0);
#pragma unroll
      for (int kz = 0; kz < N; ++kz) {
        const T2 v = col[kz * VEC];
        re[kz] = v.x;
        im[kz] = v.y;
      }
      fft_regs<N, +1>(re, im);
#pragma unroll
      for (int z = 0; z < N; ++z) col[z * VEC] = make_float2(re[z], im[z]);
    }
    // the chunk's own threads wrote its planes: a barrier among them (ids 1 ..)
    asm volatile("bar.sync %0, %1;" ::"r"(1 + chunk), "r"(CH_THREADS) : "memory");
    {  // ky pass: thread (xl, z); Q+ += w Re Im into shared memory, or keep L in re[]
      const T2* col = XB + Cfg::elem(xlt, 0, zt);
#pragma unroll
      for (int ky = 0; ky < N; ++ky) {
        const T2 v = col[ky * (RW_ * VEC)];
        re[ky] = v.x;
        im[ky] = v.y;
      }
      fft_regs<N, +1>(re, im);
      if (j < M_eff) {
        float* a = accs + (size_t)xlt * Cfg::ACC_PLANE + zt;
#pragma unroll
        for (int y = 0; y < N; ++y) a[y * N] += wj * (re[y] * im[y]);
      }
    }
    if (more) {
      // write-after-read: the chunk's threads meet (their loads of the term precede it),
      // then the chunk's first warp arrives with .release (cumulative over them) and the
      // others relaxed; the wait is in the next kx pass, before its stores
      asm volatile("bar.sync %0, %1;" ::"r"(1 + chunk), "r"(CH_THREADS) : "memory");
      if (((t % CH_THREADS) >> 5) == 0) {
        cluster_arrive_war<C>();
      } else {
        asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
      }
    }
  }
  if (nt == 0) cluster_wait_war<C>();  // a group without terms: close the forward arrive

  // the spectrum is no longer needed: free the TMEM columns
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((t >> 5) == 0) {
#pragma unroll
    for (int k = 0; k < Cfg::TMEM_SHARES; ++k)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot[k]), "r"(kTmemShare));
  }

  const int x = x_own, z = zt;
  float* acc_row = accs + (size_t)xlt * Cfg::ACC_PLANE + z;  // acc_row[y * N], this thread's (x, z) row
  if constexpr (kSplit) {
    // partial gain and loss of this group, then the last-arrival count (as collide_kernel)
    T* part;
    T* lossp;
    unsigned* arrp;
    split_scratch<T>(args, lc, G, n, part, lossp, arrp);
#pragma unroll
    for (int y = 0; y < N; ++y) {
      const int idx = (x * N + y) * N + z;
      part[(size_t)gi * n + idx] = acc_row[y * N];
      if (has_loss) lossp[idx] = re[y];
    }
    __threadfence();
    cluster_barrier<C>();
    unsigned* flag = reinterpret_cast<unsigned*>(smem_raw + Cfg::OFF_FLAG);
    if (rank == 0 && t == 0) {
      const unsigned prev = atomicAdd(arrp, 1u);
      const unsigned last = (prev == (unsigned)(G - 1)) ? 1u : 0u;
      if (last) *arrp = 0u;
#pragma unroll
      for (int q = 0; q < C; ++q) *cta_smem<C>(flag, q) = last;
    }
    cluster_barrier<C>();
    if (*flag == 0u) return;
    __threadfence();
#pragma unroll
    for (int y = 0; y < N; ++y) {
      const int idx = (x * N + y) * N + z;
      T sum = __ldcg(part + idx);
      for (int g2 = 1; g2 < G; ++g2) sum += __ldcg(part + (size_t)g2 * n + idx);
      acc_row[y * N] = sum;
      re[y] = __ldcg(lossp + idx);
    }
  }

  // ---- epilogue (float64), two sweeps over this thread's row --------------------------
  const double vx = -L + x * dv, vz = -L + z * dv;
  const TIO* fb = args.f_base ? reinterpret_cast<const TIO*>(args.f_base) + cell * n : nullptr;
  auto gval = [&](int y) {
    const int idx = (x * N + y) * N + z;
    const TIO fv = fin[idx];
    const T q = acc_row[y * N] - (T)fv * re[y];  // Q = Q+ - f L (one rounding in T)
    double gv = args.s * (double)q;
    if (args.b != 0.0) gv += args.b * (double)fv;
    if (fb) gv += args.a * (double)fb[idx];
    return gv;
  };
  double S0 = 0.0, S1 = 0.0, S2 = 0.0;
#pragma unroll
  for (int y = 0; y < N; ++y) {
    const double gv = gval(y);
    S0 += gv;
    S1 += (double)y * gv;
    S2 += (double)(y * y) * gv;
  }
  double m[5] = {S0, vx * S0, -L * S0 + dv * S1, vz * S0,
                 0.5 * ((vx * vx + vz * vz + L * L) * S0 - 2.0 * L * dv * S1 + dv * dv * S2)};
  double c5[5];
  cluster_correction<C, WARPS>(args, m, red, cell, writable, rank, t, c5);
  TIO* out = reinterpret_cast<TIO*>(args.out) + cell * n;
  bool bad = false;
  const double P0 = c5[0] + c5[1] * vx + c5[3] * vz + 0.5 * c5[4] * (vx * vx + vz * vz + L * L) - c5[2] * L;
  const double P1 = (c5[2] - c5[4] * L) * dv;
  const double P2 = 0.5 * c5[4] * dv * dv;
#pragma unroll
  for (int y = 0; y < N; ++y) {
    const double val = gval(y) + (P0 + (double)y * (P1 + (double)y * P2));
    bad |= !isfinite(val);
    if (writable) out[(x * N + y) * N + z] = (TIO)val;
  }
  if (bad) atomicOr(&g_boltz_status, kStatusNonFinite);
}

// ------------------------------------------------------------------------------------
// Two dimensions (Maxwell molecules; Sec. 3.3 dimension two, Eq. dfor0).  A cell is N
// threads (one pencil each) of a CTA that holds several cells; the cell's spectrum (in
// TMEM for float32 at N = 16, 32, in shared memory otherwise) and one N x (N+1) plane
// buffer in shared memory, the gain accumulator in registers.
// Per term: kx pass with the coefficients (thread ky, tables [term][kx][ky] read
// coalesced across the cell's threads), transposed store, ky pass (thread x) and
// Q+ += w Re Im along y.  Projection on (1, v_x, v_y, |v|^2/2) in float64 (the 5-slot
// matrix G has row and column 3 zero), two sweeps in the epilogue.
// ------------------------------------------------------------------------------------
template <typename T, int N>
struct PlaneCfg {
  using T2 = typename Vec2<T>::type;
  static constexpr int RW = N + 1;
  static constexpr size_t BUF = (size_t)N * RW;  // T2 per plane
  // float32 at N = 16, 32: each thread's spectrum pencil (2N floats) lives in TMEM (warp w:
  // lanes 32 (w % 4) .., column group w / 4), so a cell's shared memory is its plane
  // buffer and reduction rows only and two 8-cell CTAs fit on an SM
  static constexpr bool kTmemSpec = sizeof(T) == 4 && (N == 16 || N == 32);
  static constexpr size_t CELL_SMEM = (kTmemSpec ? 1 : 2) * BUF * sizeof(T2) + (size_t)(N + 1) * 10 * sizeof(double);
  static constexpr int CPB_SMEM = (int)((200u * 1024u) / CELL_SMEM);
  static constexpr int CPB = (256 / N < CPB_SMEM) ? 256 / N : CPB_SMEM;  // cells per CTA
  static constexpr int THREADS = CPB * N;
  static constexpr int MIN_BLOCKS = kTmemSpec ? 2 : 1;
  static constexpr int TMEM_SHARES = kTmemSpec ? ((THREADS / 32 + 3) / 4 * 2 * N + kTmemShare - 1) / kTmemShare : 0;
  static constexpr int GROUP_COLS = 2 * N;  // columns per group of four warps
  static constexpr size_t OFF_TSLOT = (size_t)CPB * CELL_SMEM;  // TMEM addresses (up to 4)
  static constexpr size_t SMEM = OFF_TSLOT + 16;
  static_assert(!kTmemSpec || TMEM_SHARES <= 4, "spectrum shares per CTA");
  static_assert(!kTmemSpec || TMEM_SHARES == 1 || GROUP_COLS == kTmemShare, "one share per warp group");
  static_assert(OFF_TSLOT % 8 == 0, "aligned TMEM address slots");
  static_assert(CPB >= 1, "one cell must fit");
  static_assert(N <= 32 || CPB <= 15, "one named barrier per cell (ids 1..15)");
};

template <typename T, typename TIO, int N>
__global__ void __launch_bounds__(PlaneCfg<T, N>::THREADS, PlaneCfg<T, N>::MIN_BLOCKS)
collide2d_kernel(const CollideArgs args, long long n_cells) {
  using Cfg = PlaneCfg<T, N>;
  using T2 = typename Cfg::T2;
  constexpr int RW_ = Cfg::RW;
  constexpr int n = N * N;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int ci = threadIdx.x / N, t = threadIdx.x % N;
  // The cell's threads synchronise among themselves only: the lanes of one warp for
  // N <= 32, a named barrier (id 1 + cell) of its 64 threads for N = 64.
  auto cell_sync = [&]() {
    if constexpr (N <= 32) {
      const unsigned lanes = (N == 32) ? 0xffffffffu : (((1u << N) - 1u) << ((threadIdx.x & 31) / N * N));
      __syncwarp(lanes);
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + ci), "r"(N) : "memory");
    }
  };
  constexpr bool kTmemSpec = Cfg::kTmemSpec;
  unsigned char* base = smem_raw + (size_t)ci * Cfg::CELL_SMEM;
  T2* Fh = reinterpret_cast<T2*>(base);                  // spectrum [kx][ky] (not with TMEM)
  T2* P = Fh + (kTmemSpec ? 0 : Cfg::BUF);                // plane buffer [x][ky]
  double* red = reinterpret_cast<double*>(P + Cfg::BUF);  // [N][10], then [10] cell totals
  uint32_t* spec_slots = reinterpret_cast<uint32_t*>(smem_raw + Cfg::OFF_TSLOT);
  uint32_t spec_addr = 0;
  if constexpr (kTmemSpec) {
    if ((threadIdx.x >> 5) == 0) {
#pragma unroll
      for (int k = 0; k < Cfg::TMEM_SHARES; ++k)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(spec_slots + k)),
                     "r"(kTmemShare));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int grp4 = threadIdx.x >> 7;
    const uint32_t lane_off = (uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16;
    spec_addr = (Cfg::TMEM_SHARES == 1 ? spec_slots[0] + (uint32_t)(grp4 * Cfg::GROUP_COLS) : spec_slots[grp4]) +
                lane_off;
  }

  long long lc = (long long)blockIdx.x * Cfg::CPB + ci;
  const bool in_launch = lc < n_cells;  // the last CTA may hold fewer cells
  if (!in_launch) lc = n_cells - 1;
  long long cell = lc;
  bool writable = in_launch;
  if (args.cell_idx) {
    const long long s = args.cell_idx[lc];
    const bool ok = (s >= 0 && s < args.pool_cells);
    if (!ok && in_launch && t == 0) atomicOr(&g_boltz_status, kStatusBadIndex);
    writable = writable && ok;
    cell = ok ? s : 0;
  }
  const TIO* fin = cell_input<TIO>(args, cell, t, n);  // thread t: velocity-x index t
  const T2* tab = reinterpret_cast<const T2*>(args.tab);
  const int M_eff = args.M_eff;
  const double L = args.geom.L, dv = args.geom.dv;
  T re[N], im[N], acc[N];

  // forward: y pass (thread x), then x pass (thread ky)
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
  for (int y = 0; y < N; ++y) {
    const TIO fv = fin[t * N + y];
    re[y] = (T)fv;
    im[y] = T(0);
    const double fd = to_f64(fv);
    s0 += fd;
    s1 += (double)y * fd;
    s2 += (double)(y * y) * fd;
  }
  fft_regs<N, -1>(re, im);
#pragma unroll
  for (int k = 0; k < N; ++k) P[t * RW_ + k] = mk2<T>(re[k], im[k]);
  cell_sync();
#pragma unroll
  for (int x = 0; x < N; ++x) {
    const T2 v = P[x * RW_ + t];
    re[x] = v.x;
    im[x] = v.y;
  }
  fft_regs<N, -1>(re, im);
  {
    const T scale = T(1) / T(n);
#pragma unroll
    for (int kx = 0; kx < N; ++kx) {
      const bool z0 = (kx == N / 2) || (t == N / 2);
      if constexpr (kTmemSpec) {
        re[kx] = z0 ? T(0) : re[kx] * scale;
        im[kx] = z0 ? T(0) : im[kx] * scale;
      } else {
        Fh[kx * RW_ + t] = z0 ? mk2<T>(T(0), T(0)) : mk2<T>(re[kx] * scale, im[kx] * scale);
      }
    }
    if constexpr (kTmemSpec) {
#pragma unroll
      for (int c = 0; c < N; c += 16) {
        tmem_st16(spec_addr + c, reinterpret_cast<const float*>(re) + c);
        tmem_st16(spec_addr + N + c, reinterpret_cast<const float*>(im) + c);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
  }
#pragma unroll
  for (int y = 0; y < N; ++y) acc[y] = T(0);
  cell_sync();

  for (int j = 0; j <= M_eff; ++j) {
    const T wj = (j < M_eff) ? (T)args.w[j] : T(0);
    const T2* tj = tab + (size_t)j * n + t;
    if constexpr (kTmemSpec) {
#pragma unroll
      for (int c = 0; c < N; c += 16) {
        tmem_ld16(spec_addr + c, reinterpret_cast<float*>(re) + c);
        tmem_ld16(spec_addr + N + c, reinterpret_cast<float*>(im) + c);
      }
      tmem_wait_ld<N>(reinterpret_cast<float*>(re));
      tmem_wait_ld<N>(reinterpret_cast<float*>(im));
    }
#pragma unroll
    for (int kx = 0; kx < N; ++kx) {
      T2 c;
      if constexpr (kTmemSpec) {
        c = mk2<T>(re[kx], im[kx]);
      } else {
        c = Fh[kx * RW_ + t];
      }
      const T2 ab = __ldg(tj + kx * N);
      re[kx] = ab.x * c.x - ab.y * c.y;
      im[kx] = ab.x * c.y + ab.y * c.x;
    }
    fft_regs<N, +1>(re, im);
#pragma unroll
    for (int x = 0; x < N; ++x) P[x * RW_ + t] = mk2<T>(re[x], im[x]);
    cell_sync();
#pragma unroll
    for (int ky = 0; ky < N; ++ky) {
      const T2 v = P[t * RW_ + ky];
      re[ky] = v.x;
      im[ky] = v.y;
    }
    fft_regs<N, +1>(re, im);
    if (j < M_eff) {
#pragma unroll
      for (int y = 0; y < N; ++y) acc[y] += wj * (re[y] * im[y]);
    }
    cell_sync();  // the next term overwrites P
  }
  // re[] holds the loss multiplier L along y of row x = t
  if constexpr (kTmemSpec) {
    // the spectrum is no longer needed: free its TMEM columns
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
#pragma unroll
      for (int k = 0; k < Cfg::TMEM_SHARES; ++k)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(spec_slots[k]), "r"(kTmemShare));
    }
  }

  const int x = t;
  const double vx = -L + x * dv;
  const TIO* fb = args.f_base ? reinterpret_cast<const TIO*>(args.f_base) + cell * n : nullptr;
  // g = s Q + b f (+ a f_base) along this row; Q = Q+ - f L rounded once in T
  auto qval = [&](int y) { return to_f64(acc[y] - (T)fin[x * N + y] * re[y]); };
  // Phi g over the row: the f part is b times the forward pass's sums s0, s1, s2 of the
  // same row, so only Q (and f_base) is summed here (the FP64 pipe bounds this kernel)
  double Q0 = 0.0, Q1 = 0.0, Q2 = 0.0, F0 = 0.0, F1 = 0.0, F2 = 0.0;
#pragma unroll
  for (int y = 0; y < N; ++y) {
    const double qv = qval(y);
    Q0 += qv;
    Q1 += (double)y * qv;
    Q2 += (double)(y * y) * qv;
    if (fb) {
      const double bv = to_f64(fb[x * N + y]);
      F0 += bv;
      F1 += (double)y * bv;
      F2 += (double)(y * y) * bv;
    }
  }
  const double S0 = args.s * Q0 + args.b * s0 + args.a * F0;
  const double S1 = args.s * Q1 + args.b * s1 + args.a * F1;
  const double S2 = args.s * Q2 + args.b * s2 + args.a * F2;
  // this row's share of Phi g and Phi f (targets), v_y = -L + y dv; slot 3 (v_z) is zero
  {
    double* r = red + t * 10;
    r[0] = S0;
    r[1] = vx * S0;
    r[2] = -L * S0 + dv * S1;
    r[3] = 0.0;
    r[4] = 0.5 * ((vx * vx + L * L) * S0 - 2.0 * L * dv * S1 + dv * dv * S2);
    r[5] = s0;
    r[6] = vx * s0;
    r[7] = -L * s0 + dv * s1;
    r[8] = 0.0;
    r[9] = 0.5 * ((vx * vx + L * L) * s0 - 2.0 * L * dv * s1 + dv * dv * s2);
  }
  cell_sync();
  double* tot = red + N * 10;
  if (t < 10) {
    double v = 0.0;
    for (int q = 0; q < N; ++q) v += red[q * 10 + t];
    tot[t] = v;
  }
  cell_sync();
  double c5[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (args.project) {
    double tgt[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (args.compute_targets) {
#pragma unroll
      for (int r = 0; r < 5; ++r) tgt[r] = tot[5 + r];
      if (args.Utgt && writable && t == 0) {
#pragma unroll
        for (int r = 0; r < 5; ++r) args.Utgt[cell * 5 + r] = tgt[r];
      }
    } else if (args.Utgt) {
#pragma unroll
      for (int r = 0; r < 5; ++r) tgt[r] = args.Utgt[cell * 5 + r];
    }
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      double v = 0.0;
#pragma unroll
      for (int k = 0; k < 5; ++k) v += args.geom.G[r * 5 + k] * (tgt[k] - tot[k]);
      c5[r] = v;
    }
  }
  TIO* out = reinterpret_cast<TIO*>(args.out) + cell * n;
  bool bad = false;
  // Phi^T c at (vx, vy) = P0 + R(y), R(y) = y (P1 + y P2) the same for every row of the
  // cell: thread t writes R(t) over its row sums (read above), the row adds its own P0
  const double P0 = c5[0] + c5[1] * vx + 0.5 * c5[4] * (vx * vx + L * L) - c5[2] * L;
  const double P1 = (c5[2] - c5[4] * L) * dv;
  const double P2 = 0.5 * c5[4] * dv * dv;
  red[t] = (double)t * (P1 + (double)t * P2);
  cell_sync();
#pragma unroll
  for (int y = 0; y < N; ++y) {
    const int idx = x * N + y;
    double val = fma(args.b, to_f64(fin[idx]), P0 + red[y]);
    if (fb) val = fma(args.a, to_f64(fb[idx]), val);
    val = fma(args.s, qval(y), val);
    bad |= !isfinite(val);
    if (writable) out[idx] = from_f64<TIO>(val);
  }
  if (bad && writable) atomicOr(&g_boltz_status, kStatusNonFinite);
}

// ------------------------------------------------------------------------------------
// launchers (instantiated by the unit that dispatches them)
// ------------------------------------------------------------------------------------

static inline boltz_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return BOLTZ_ECUDA;
}

// Dynamic shared memory to launch a kernel with that holds `held` TMEM columns per CTA
// in `shares` allocations of kTmemShare columns (held = 0: none; held above shares x
// kTmemShare: one larger allocation that must not share the SM with a TMEM holder), given
// the `smem` bytes it uses.  With P bytes of shared memory per SM and r bytes kept by the
// hardware per CTA, a CTA of k shares takes at least k (P/9 + 1) - r bytes, so no nine
// shares ever fit; a CTA holding a larger allocation takes enough that not even one
// sharing CTA fits beside it.
static inline boltz_status tmem_launch_smem(int held, size_t smem, int dev, size_t* out, int shares = 1) {
  *out = smem;
  if (held == 0) return BOLTZ_OK;
  int per_sm = 0, reserved = 0, optin = 0;
  cudaError_t e;
  if ((e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return cuda_fail(e, "shared memory attributes");
  const size_t P = (size_t)per_sm, r = (size_t)reserved;
  const size_t share = P / 9 + 1 - (r < P / 9 + 1 ? r : P / 9);
  // a CTA holding k shares takes (need + r) >= k (P / 9 + 1): at most 8 shares per SM
  size_t need = shares * (P / 9 + 1) > r ? shares * (P / 9 + 1) - r : share;
  if (held > shares * kTmemShare) need = P + 1 - share - 2 * r;  // (need + r) + (share + r) > P
  if (need > *out) *out = need;
  if (*out > (size_t)optin) {
    set_error("shared memory reservation for tensor memory exceeds the per-block limit");
    return BOLTZ_EUNSUPPORTED;
  }
  return BOLTZ_OK;
}

template <typename T, typename TIO, int N, int C, int TC = kTcNone>
static boltz_status launch_impl(const CollideArgs& a, int64_t n_cells, cudaStream_t st) {
  using Cfg = CollideCfg<T, N, C, TC>;
  const bool split = a.groups > 1;
  void (*kern)(const CollideArgs);
  if constexpr (TC != kTcNone) {
    kern = collide_kernel<T, TIO, N, C, false, TC>;  // no term groups with tensor-core transforms
  } else {
    kern = split ? collide_kernel<T, TIO, N, C, true> : collide_kernel<T, TIO, N, C, false>;
  }
  // function attributes are per device: set them once per (instantiation, device), and
  // check once that a cluster of this size can be scheduled at all
  static std::atomic<unsigned long long> prepared[2], unschedulable[2];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  const unsigned long long bit = 1ull << (dev & 63);
  size_t smem = Cfg::SMEM;
  const boltz_status ss = tmem_launch_smem(Cfg::TMEM_HELD, Cfg::SMEM, dev, &smem,
                                           Cfg::TMEM_SHARES > 1 ? Cfg::TMEM_SHARES : 1);
  if (ss != BOLTZ_OK) return ss;
  if (dev >= 64 || !(prepared[split].load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    if (C > 1) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
      cudaLaunchConfig_t q = {};
      q.gridDim = dim3(C, 1, 1);
      q.blockDim = dim3(Cfg::THREADS, 1, 1);
      q.dynamicSmemBytes = smem;
      cudaLaunchAttribute qa[1];
      qa[0].id = cudaLaunchAttributeClusterDimension;
      qa[0].val.clusterDim.x = C;
      qa[0].val.clusterDim.y = 1;
      qa[0].val.clusterDim.z = 1;
      q.attrs = qa;
      q.numAttrs = 1;
      int clusters = 0;
      e = cudaOccupancyMaxActiveClusters(&clusters, kern, &q);
      if (e != cudaSuccess || clusters < 1) {
        cudaGetLastError();
        if (dev < 64) unschedulable[split].fetch_or(bit, std::memory_order_release);
      }
    }
    if (dev < 64) prepared[split].fetch_or(bit, std::memory_order_release);
  }
  if (dev < 64 && (unschedulable[split].load(std::memory_order_acquire) & bit)) {
    set_error("a thread-block cluster of this size cannot be scheduled on this device");
    return BOLTZ_EUNSUPPORTED;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_cells * a.groups * C), 1, 1);
  cfg.blockDim = dim3(Cfg::THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (C > 1) ? 1 : 0;
  e = cudaLaunchKernelEx(&cfg, kern, a);
  if (e != cudaSuccess) return cuda_fail(e, "collide launch");
  return BOLTZ_OK;
}

template <typename TIO, int N, int C>
static boltz_status launch_large_impl(const CollideArgs& a, int64_t n_cells, cudaStream_t st) {
  using Cfg = LargeCfg<N, C>;
  const bool split = a.groups > 1;
  auto kern = split ? collide_large_kernel<TIO, N, C, true> : collide_large_kernel<TIO, N, C, false>;
  static std::atomic<unsigned long long> prepared[2], unschedulable[2];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  const unsigned long long bit = 1ull << (dev & 63);
  size_t smem = Cfg::SMEM;
  const boltz_status ss = tmem_launch_smem(Cfg::TMEM_SHARES * kTmemShare, Cfg::SMEM, dev, &smem, Cfg::TMEM_SHARES);
  if (ss != BOLTZ_OK) return ss;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  if (dev >= 64 || !(prepared[split].load(std::memory_order_acquire) & bit)) {
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
      return cuda_fail(e, "cudaFuncSetAttribute");
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3(C, 1, 1);
    q.blockDim = dim3(Cfg::THREADS, 1, 1);
    q.dynamicSmemBytes = smem;
    q.attrs = attr;
    q.numAttrs = 1;
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, kern, &q);
    if (e != cudaSuccess || clusters < 1) {
      cudaGetLastError();
      if (dev < 64) unschedulable[split].fetch_or(bit, std::memory_order_release);
    }
    if (dev < 64) prepared[split].fetch_or(bit, std::memory_order_release);
  }
  if (dev < 64 && (unschedulable[split].load(std::memory_order_acquire) & bit)) {
    set_error("a thread-block cluster of this size cannot be scheduled on this device");
    return BOLTZ_EUNSUPPORTED;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_cells * a.groups * C), 1, 1);
  cfg.blockDim = dim3(Cfg::THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, a);
  if (e != cudaSuccess) return cuda_fail(e, "collide launch");
  return BOLTZ_OK;
}

template <typename T, typename TIO, int N>
static boltz_status launch2d_impl(const CollideArgs& a, int64_t n_cells, cudaStream_t st) {
  using Cfg = PlaneCfg<T, N>;
  auto kern = collide2d_kernel<T, TIO, N>;
  static std::atomic<unsigned long long> prepared{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  const unsigned long long bit = 1ull << (dev & 63);
  size_t smem = Cfg::SMEM;
  const boltz_status ss = tmem_launch_smem(Cfg::TMEM_SHARES * kTmemShare, Cfg::SMEM, dev, &smem,
                                           Cfg::TMEM_SHARES > 1 ? Cfg::TMEM_SHARES : 1);
  if (ss != BOLTZ_OK) return ss;
  if (dev >= 64 || !(prepared.load(std::memory_order_acquire) & bit)) {
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return cuda_fail(e, "cudaFuncSetAttribute");
    if (dev < 64) prepared.fetch_or(bit, std::memory_order_release);
  }
  const long long blocks = (n_cells + Cfg::CPB - 1) / Cfg::CPB;
  kern<<<(unsigned)blocks, Cfg::THREADS, smem, st>>>(a, (long long)n_cells);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "collide2d launch");
  return BOLTZ_OK;
}

// Per-unit services: the twiddle constants and the status word are per translation unit.
#define BOLTZ_UNIT_SERVICES(TAG)                                                                  \
  cudaError_t unit_upload_twiddles_##TAG(const TwiddleTables& t) {                                 \
    cudaError_t e;                                                                                \
    if ((e = cudaMemcpyToSymbol(c_twc64, t.c64, sizeof(t.c64))) != cudaSuccess) return e;        \
    if ((e = cudaMemcpyToSymbol(c_tws64, t.s64, sizeof(t.s64))) != cudaSuccess) return e;        \
    if ((e = cudaMemcpyToSymbol(c_twl64, t.l64, sizeof(t.l64))) != cudaSuccess) return e;        \
    if ((e = cudaMemcpyToSymbol(c_twm64, t.m64, sizeof(t.m64))) != cudaSuccess) return e;        \
    if ((e = cudaMemcpyToSymbol(c_twr64, t.r64, sizeof(t.r64))) != cudaSuccess) return e;        \
    if ((e = cudaMemcpyToSymbol(c_twc32, t.c32, sizeof(t.c32))) != cudaSuccess) return e;        \
    if ((e = cudaMemcpyToSymbol(c_tws32, t.s32, sizeof(t.s32))) != cudaSuccess) return e;        \
    if ((e = cudaMemcpyToSymbol(c_twl32, t.l32, sizeof(t.l32))) != cudaSuccess) return e;        \
    if ((e = cudaMemcpyToSymbol(c_twm32, t.m32, sizeof(t.m32))) != cudaSuccess) return e;        \
    return cudaMemcpyToSymbol(c_twr32, t.r32, sizeof(t.r32));                                    \
  }                                                                                               \
  cudaError_t unit_read_clear_status_##TAG(unsigned* value) {                                     \
    unsigned v = 0, zero = 0;                                                                     \
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_boltz_status, sizeof(v));                          \
    if (e != cudaSuccess) return e;                                                               \
    *value |= v;                                                                                  \
    return cudaMemcpyToSymbol(g_boltz_status, &zero, sizeof(zero));                               \
  }

}  // namespace boltz
