// One CTA per cell at N = 32 (float32 transforms): the whole cell on one SM, no cluster.
//
// Paper: arxiv 1608.08009, Sec. 3.3 (the operator: one forward transform of f, per
// separated term one packed complex inverse transform whose real and imaginary parts are
// the two factors of the gain, the loss transform), Sec. 3.2 (projection), Sec. 3.1
// Eq. f_coll (update), Sec. 4.2 (the per-cell loop).  Same arithmetic as collide_kernel in
// another order of the transform stages; included by the unit that dispatches it, after
// collide_kernels.cuh.
//
// A 32^3 float32 cell does not fit an SM whole: its spectrum, its gain accumulator and one
// complex field of an inverse transform are 256 + 128 + 256 KB.  So:
//  * Spectrum: f is real, so fhat(-k) = conj fhat(k) and half of it is kept: the pencils
//    (ky, kz) with ky < 16 along kx, in TMEM (thread (ky, kz) = warp ky, lane kz, 64
//    columns: fhat(g), fhat(g + 16) for g = 0..15 as re, im, re, im).  Thread (ky, kz)
//    also forms the pencil (-ky, -kz) from its own: alpha and alpha' are even, so the
//    coefficients of (-ky, -kz) are those of (ky, kz) with kx reversed.
//  * Gain accumulator: the other 256 TMEM columns (thread (m, z) = warp m, lane z holds
//    the y-rows of x = 2 m and 2 m + 1 at z).
//  * One inverse transform in two halves of its output: x = 2 m + h, h = 0, 1.  One
//    radix-2 decimation-in-frequency step along kx, u_h(k) = w^{hk} (c(k) + (-1)^h
//    c(k + 16)), w = exp(2 pi i / 32), leaves a 16-point transform along kx per half, and
//    the half field [m][ky][kz] (16 x 32 x 33 float2, 132 KB) fits shared memory.  Each
//    half forms the coefficients (alpha + i alpha') fhat again: 1.45 M instead of 1.37 M
//    FP32 instructions per cell and term.
//  * Per half: P1 (thread (ky, kz): coefficients, u_h, two 16-point transforms, stores of
//    both pencils' outputs), a CTA barrier, P2 (warp m: the kz pass of plane m), P3 (warp
//    m: the ky pass of plane m and the gain update in TMEM), a CTA barrier.  Nothing
//    leaves the SM: no cluster, no distributed shared memory.
// Twiddles, tables and weights are float32; moments, projection and update float64, with
// the float <-> double conversions on the integer pipes (exact, to_f64 / from_f64): with
// every warp of the SM in the same cell, the float64 phases of a cell do not overlap
// another cell's float32 work, and the hardware conversions issue to the FP64 pipe.
#pragma once

#include "collide_kernels.cuh"

namespace boltz {

struct SoloCfg {
  static constexpr int N = 32;
  static constexpr int HN = N / 2;          // x-values per half of the output
  static constexpr int THREADS = 512;       // 16 warps
  static constexpr int WARPS = THREADS / 32;
  static constexpr int RS = N + 1;          // float2 per row: odd, so rows and columns are conflict-free
  static constexpr int PLANE = N * RS;      // float2 per plane m of the half field [m][ky][kz]
  static constexpr int SX = HN * RS;        // float2 per x of the forward buffer [x][ky < 16][z]
  static constexpr size_t FIELD = (size_t)HN * PLANE;
  static_assert((size_t)N * SX == FIELD, "the forward buffer and the half field share their bytes");
  static constexpr size_t OFF_RED = FIELD * sizeof(float2);
  // red: [WARPS][10] warp partials (Phi g, then Phi f_in), then [10] totals
  static constexpr size_t OFF_MG = OFF_RED + (size_t)(WARPS + 1) * 10 * sizeof(double);
  // [5][THREADS] each thread's share of Phi g, summed over its two rows in shared memory
  // (held in registers across the angular loop it would cost ten of them there)
  static constexpr size_t OFF_TSLOT = OFF_MG + (size_t)5 * THREADS * sizeof(double);
  static constexpr size_t SMEM = OFF_TSLOT + 16;
  static constexpr int TMEM_COLS = 512;     // spectrum half (columns 0..255), accumulator (256..511)
  static constexpr int ACC_COL = 256;
  static_assert(SMEM <= 232448, "shared memory per CTA");
};

template <typename TIO>
__global__ void __launch_bounds__(SoloCfg::THREADS, 1) collide_solo_kernel(const CollideArgs args) {
  using Cfg = SoloCfg;
  constexpr int N = Cfg::N, HN = Cfg::HN, RS = Cfg::RS, PLANE = Cfg::PLANE, SX = Cfg::SX, WARPS = Cfg::WARPS;
  constexpr int n = N * N * N;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* Wb = reinterpret_cast<float2*>(smem_raw);
  double* red = reinterpret_cast<double*>(smem_raw + Cfg::OFF_RED);
  double* mgs = reinterpret_cast<double*>(smem_raw + Cfg::OFF_MG) + threadIdx.x;  // mgs[r * THREADS]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem_raw + Cfg::OFF_TSLOT);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

  // Slot of this cell; an index outside [0, pool_cells) is reported, reads slot 0 and
  // writes nothing.
  long long cell = blockIdx.x;
  bool writable = true;
  if (args.cell_idx) {
    const long long s = args.cell_idx[cell];
    writable = (s >= 0 && s < args.pool_cells);
    if (!writable && t == 0) atomicOr(&g_boltz_status, kStatusBadIndex);
    cell = writable ? s : 0;
  }

  // All 512 TMEM columns (the launch reserves enough shared memory that no other TMEM
  // holder shares the SM, so the allocation never waits).
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(Cfg::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tm = *tslot;
  // warp w reaches lanes 32 (w % 4) .. + 31; the four warps of one lane range use column
  // groups w / 4.  Every thread touches only its own lane: no TMEM data crosses threads.
  const uint32_t lane_base = tm + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t spec = lane_base + (uint32_t)((warp >> 2) * 64);
  const uint32_t accb = lane_base + (uint32_t)(Cfg::ACC_COL + (warp >> 2) * 64);

  const double L = args.geom.L, dv = args.geom.dv;
  const float2* tab = reinterpret_cast<const float2*>(args.tab);
  const int M_eff = args.M_eff;
  float re[N], im[N];

  // ---- forward transform: pass along y of two real rows packed as one complex row ----
  {
    const int x = t >> 4, z0 = t & 15;  // rows (x, z0) and (x, z0 + 16)
    const TIO* fin = cell_input<TIO>(args, cell, x, n);
    double s0p = 0.0, s1p = 0.0, s2p = 0.0, s0q = 0.0, s1q = 0.0, s2q = 0.0;
#pragma unroll
    for (int y = 0; y < N; ++y) {
      const TIO p = fin[(x * N + y) * N + z0], q = fin[(x * N + y) * N + z0 + HN];
      re[y] = (float)p;
      im[y] = (float)q;
      if (args.compute_targets) {
        const double pd = to_f64(p), qd = to_f64(q);
        s0p += pd;
        s1p += (double)y * pd;
        s2p += (double)(y * y) * pd;
        s0q += qd;
        s1q += (double)y * qd;
        s2q += (double)(y * y) * qd;
      }
    }
    if (args.compute_targets) {
      // Phi f over the two rows, v = (-L + x dv, -L + y dv, -L + z dv)
      const double vx = -L + x * dv, vp = -L + z0 * dv, vq = -L + (z0 + HN) * dv;
      const double yyp = L * L * s0p - 2.0 * L * dv * s1p + dv * dv * s2p;
      const double yyq = L * L * s0q - 2.0 * L * dv * s1q + dv * dv * s2q;
      double m[5] = {s0p + s0q, vx * (s0p + s0q), (-L * s0p + dv * s1p) + (-L * s0q + dv * s1q),
                     vp * s0p + vq * s0q,
                     0.5 * ((vx * vx + vp * vp) * s0p + yyp + (vx * vx + vq * vq) * s0q + yyq)};
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        const double v = warp_sum(m[r]);
        if (lane == 0) red[warp * 10 + 5 + r] = v;
      }
    }
    fft_regs<N, -1>(re, im);
    // Z = P + i Q with P, Q the transforms of the real rows: P(k) = (Z(k) + conj Z(-k)) / 2,
    // Q(k) = (Z(k) - conj Z(-k)) / 2i; kept for ky < 16 (ky = 16 is removed anyway)
    float2* row = Wb + (size_t)x * SX + z0;
#pragma unroll
    for (int k = 0; k < HN; ++k) {
      const int kn = (N - k) & (N - 1);
      const float zr = re[k], zi = im[k], wr = re[kn], wi = im[kn];
      row[k * RS] = make_float2(0.5f * (zr + wr), 0.5f * (zi - wi));
      row[k * RS + HN] = make_float2(0.5f * (zi + wi), -0.5f * (zr - wr));
    }
  }
  __syncthreads();
  // ---- pass along z: thread (x, ky) -----------------------------------------------------
  {
    const int x = t >> 4, ky = t & 15;
    float2* row = Wb + (size_t)x * SX + ky * RS;
#pragma unroll
    for (int z = 0; z < N; ++z) {
      const float2 v = row[z];
      re[z] = v.x;
      im[z] = v.y;
    }
    fft_regs<N, -1>(re, im);
#pragma unroll
    for (int k = 0; k < N; ++k) row[k] = make_float2(re[k], im[k]);
  }
  __syncthreads();
  // ---- pass along x: thread (ky, kz) = (warp, lane); the spectrum half into TMEM ---------
  {
    const int ky = warp, kz = lane;
    const float2* col = Wb + ky * RS + kz;
#pragma unroll
    for (int x = 0; x < N; ++x) {
      const float2 v = col[(size_t)x * SX];
      re[x] = v.x;
      im[x] = v.y;
    }
    fft_regs<N, -1>(re, im);
    const float scale = 1.f / (float)n;
    // every mode with a component -N/2 is removed: kz = 16 (the whole pencil), kx = 16
    // (ky < 16 here; the row ky = 16 is never formed)
    const bool nyq = (kz == HN);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float w16[16];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int g = 4 * c + q;
        w16[4 * q + 0] = nyq ? 0.f : re[g] * scale;
        w16[4 * q + 1] = nyq ? 0.f : im[g] * scale;
        w16[4 * q + 2] = (nyq || g == 0) ? 0.f : re[g + HN] * scale;
        w16[4 * q + 3] = (nyq || g == 0) ? 0.f : im[g + HN] * scale;
      }
      tmem_st16(spec + 16 * c, w16);
    }
    // the gain accumulator starts at zero
    float z16[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) z16[q] = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) tmem_st16(accb + 16 * c, z16);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  __syncthreads();  // the x pass has read the forward buffer: the half field may be written
  // the row ky = 16 of every plane stays zero: no pencil writes it, and its kz pass maps
  // zeros to zeros
  Wb[(size_t)(t >> 5) * PLANE + HN * RS + (t & 31)] = make_float2(0.f, 0.f);

  // ---- angular loop: per term two halves of one packed complex inverse transform -------
  // P1 roles.  Pencil A = (ky, kz) is the thread's own, B = (-ky, -kz) its mirror.  Every
  // (ky', kz') off the removed row ky' = 16 and column kz' = 16 is formed exactly once: by
  // A for ky' in 1..15, by the mirror of (32 - ky', -kz') for ky' in 17..31, and in the row
  // ky' = 0 by A of (0, kz') for kz' in 0..15 and by B of (0, 32 - kz') for kz' in 17..31.
  const int ky = warp, kz = lane;
  const bool doA = (kz != HN) && !(ky == 0 && kz > HN);
  const bool doB = doA && !(ky == 0 && kz == 0);
  const int kyB = (N - ky) & (N - 1), kzB = (N - kz) & (N - 1);
  const int mp = warp, zp = lane;             // P2 / P3: plane m = warp; ky (P2) or z (P3) = lane
  // g = s Q + b f (+ a f_base, added by the caller) in float64; the usual step (b = 1)
  // as one fused multiply-add
  const bool b_one = (args.b == 1.0);
  // With the targets computed here (Phi f_in summed by the forward pass) and no f_base,
  // Phi g = s Phi Q + b Phi f_in: the loss pass then sums Q alone, one float64 operation a
  // point fewer
  const bool q_sums = args.compute_targets && !args.f_base;
  auto gval = [&](float qv, TIO fv) -> double {
    const double qd = to_f64(qv);
    if (b_one) return fma(args.s, qd, to_f64(fv));
    double gv = args.s * qd;
    if (args.b != 0.0) gv += args.b * to_f64(fv);
    return gv;
  };
  // the first coefficient pair of the next half's P1, loaded before the barrier that
  // precedes it, so that the L2 latency overlaps the barrier
  float2 pf[2];
  {
    const float2* t0 = tab + (size_t)ky * N * N + kz;
    pf[0] = __ldg(t0);
    pf[1] = __ldg(t0 + HN * N);
  }
  for (int j = 0; j <= M_eff; ++j) {
    const float wj = (j < M_eff) ? (float)args.w[j] : 0.f;
    // coefficients of term j (entry M_eff: (D, 0)) along kx at (ky, kz): tj[kx N]
    const float2* tj = tab + (size_t)j * n + (size_t)ky * N * N + kz;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      // ---- P1: u_h of A and B, 16-point inverse transforms, outputs x = 2 m + h ----------
      // Every lane runs the loads and the arithmetic (the TMEM loads are warp-collective
      // .sync.aligned instructions; the coefficients exist for every lane); only the stores
      // depend on the lane's role.
      {
        float ar[HN], ai[HN], br[HN], bi[HN];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float fv[16];
          tmem_ld16(spec + 16 * c, fv);
          tmem_wait_ld16(fv);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int g = 4 * c + q;  // fhat(g) and fhat(g + 16) of A; fhat(16) = 0
            const float f1r = fv[4 * q], f1i = fv[4 * q + 1], f2r = fv[4 * q + 2], f2i = fv[4 * q + 3];
            const float2 T1 = (g == 0) ? pf[0] : __ldg(tj + g * N);
            const float2 T2 = (g == 0) ? pf[1] : __ldg(tj + (g + HN) * N);
            const float sg = h ? -1.f : 1.f;
            // A at k = g: T1 f1 + (-1)^h T2 f2
            const float uar = T1.x * f1r - T1.y * f1i + sg * (T2.x * f2r - T2.y * f2i);
            const float uai = T1.x * f1i + T1.y * f1r + sg * (T2.x * f2i + T2.y * f2r);
            // B at k = 16 - g (g = 0: k = 0): its coefficient at k is A's at -k and its
            // spectrum conj fhat_A(-k); -k = g + 16 and -(k + 16) = g (g = 0: the roles swap,
            // and the second term vanishes with fhat(16))
            const float sb = (g == 0) ? 1.f : sg;
            const float ubr = T2.x * f2r + T2.y * f2i + sb * (T1.x * f1r + T1.y * f1i);
            const float ubi = T2.y * f2r - T2.x * f2i + sb * (T1.y * f1r - T1.x * f1i);
            const int kb = (HN - g) & (HN - 1);
            if (h) {
              twiddle<+1, float>(g * (kTw / N), uar, uai, ar[g], ai[g]);
              twiddle<+1, float>(kb * (kTw / N), ubr, ubi, br[kb], bi[kb]);
            } else {
              ar[g] = uar;
              ai[g] = uai;
              br[kb] = ubr;
              bi[kb] = ubi;
            }
          }
        }
        fft_regs<HN, +1>(ar, ai);
        fft_regs<HN, +1>(br, bi);
        if (doA) {
          float2* dA = Wb + ky * RS + kz;
#pragma unroll
          for (int m = 0; m < HN; ++m) dA[m * PLANE] = make_float2(ar[m], ai[m]);
        }
        if (doB) {
          float2* dB = Wb + kyB * RS + kzB;
#pragma unroll
          for (int m = 0; m < HN; ++m) dB[m * PLANE] = make_float2(br[m], bi[m]);
        }
        if (kz == HN) {
          // the column kz = 16 is removed: zero it again (the last kz pass wrote z = 16 there)
          float2* d0 = Wb + ky * RS + HN;
          float2* d1 = Wb + (ky + HN) * RS + HN;
#pragma unroll
          for (int m = 0; m < HN; ++m) {
            d0[m * PLANE] = make_float2(0.f, 0.f);
            d1[m * PLANE] = make_float2(0.f, 0.f);
          }
        }
      }
      __syncthreads();
      // ---- P2: pass along kz of plane mp, lane = ky ---------------------------------------
      {
        float2* row = Wb + mp * PLANE + lane * RS;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const float2 v = row[k];
          re[k] = v.x;
          im[k] = v.y;
        }
        fft_regs<N, +1>(re, im);
#pragma unroll
        for (int z = 0; z < N; ++z) row[z] = make_float2(re[z], im[z]);
      }
      __syncwarp();  // plane mp is this warp's alone
      // ---- P3: pass along ky of plane mp, lane = z; the gain update ------------------------
      {
        const float2* col = Wb + mp * PLANE + zp;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const float2 v = col[k * RS];
          re[k] = v.x;
          im[k] = v.y;
        }
        fft_regs<N, +1>(re, im);
        const uint32_t acol = accb + (uint32_t)(h * 32);  // y-row of x = 2 mp + h at z = zp
        const int x = 2 * mp + h;
        if (j < M_eff) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            float a16[16];
            tmem_ld16(acol + 16 * c, a16);
            tmem_wait_ld16(a16);
#pragma unroll
            for (int q = 0; q < 16; ++q) a16[q] += wj * (re[16 * c + q] * im[16 * c + q]);
            tmem_st16(acol + 16 * c, a16);
          }
        } else {
          // loss: re[] is L(v) along y.  Q = Q+ - f L (one rounding in float) replaces the
          // gain; the row's share of Phi g, g = s Q + b f (+ a f_base), in float64
          const TIO* fin = cell_input<TIO>(args, cell, x, n);
          const TIO* fb = args.f_base ? reinterpret_cast<const TIO*>(args.f_base) + cell * n : nullptr;
          double S0 = 0.0, S1 = 0.0, S2 = 0.0;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            float a16[16];
            tmem_ld16(acol + 16 * c, a16);
            tmem_wait_ld16(a16);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const int y = 16 * c + q;
              const int idx = (x * N + y) * N + zp;
              const TIO fv = fin[idx];
              const float qv = a16[q] - (float)fv * re[y];
              a16[q] = qv;
              double gv;
              if (q_sums) {
                gv = to_f64(qv);
              } else {
                gv = gval(qv, fv);
                if (fb) gv += args.a * to_f64(fb[idx]);
              }
              S0 += gv;
              S1 += (double)y * gv;
              S2 += (double)(y * y) * gv;
            }
            tmem_st16(acol + 16 * c, a16);
          }
          const double vx = -L + x * dv, vz = -L + zp * dv;
          const double m5[5] = {S0, vx * S0, -L * S0 + dv * S1, vz * S0,
                                0.5 * ((vx * vx + vz * vz + L * L) * S0 - 2.0 * L * dv * S1 + dv * dv * S2)};
#pragma unroll
          for (int r = 0; r < 5; ++r) mgs[r * Cfg::THREADS] = (h ? mgs[r * Cfg::THREADS] : 0.0) + m5[r];
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      }
      if (!h || j < M_eff) {  // the next half: (j, 1) or (j + 1, 0)
        const float2* tn = h ? tj + n : tj;
        pf[0] = __ldg(tn);
        pf[1] = __ldg(tn + HN * N);
      }
      __syncthreads();  // the planes are read: the next P1 may overwrite them
    }
  }

  // ---- projection (Sec. 3.2, Eq. minim1) and output: thread (mp, zp), rows x = 2 mp + h --
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const double v = warp_sum(mgs[r * Cfg::THREADS]);
    if (lane == 0) red[warp * 10 + r] = v;
  }
  __syncthreads();
  if (t < 10) {
    double v = 0.0;
    for (int w = 0; w < WARPS; ++w) v += red[w * 10 + t];
    red[WARPS * 10 + t] = v;  // [0..4] Phi g, [5..9] Phi f_in
  }
  __syncthreads();
  double c5[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (args.project) {
    const double* sums = red + WARPS * 10;
    double tot[5];  // Phi g
#pragma unroll
    for (int r = 0; r < 5; ++r) tot[r] = q_sums ? args.s * sums[r] + args.b * sums[5 + r] : sums[r];
    double tgt[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (args.compute_targets) {
#pragma unroll
      for (int r = 0; r < 5; ++r) tgt[r] = sums[5 + r];
      if (args.Utgt && writable) {
#pragma unroll
        for (int r = 0; r < 5; ++r)
          if (t == r) args.Utgt[cell * 5 + r] = tgt[r];  // constant register index
      }
    } else if (args.Utgt) {
#pragma unroll
      for (int r = 0; r < 5; ++r) tgt[r] = args.Utgt[cell * 5 + r];
    }
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 5; ++k) s += args.geom.G[r * 5 + k] * (tgt[k] - tot[k]);
      c5[r] = s;
    }
  }
  // R(y) = y (P1 + y P2), the y-part of Phi^T c, the same for every row of the cell:
  // tabulated once in the (no longer used) warp partials
  double* Ry = red;
  if (t < N) {
    const double P1 = (c5[2] - c5[4] * L) * dv, P2 = 0.5 * c5[4] * dv * dv;
    Ry[t] = (double)t * (P1 + (double)t * P2);
  }
  __syncthreads();
  TIO* out = reinterpret_cast<TIO*>(args.out) + cell * n;
  const TIO* fb = args.f_base ? reinterpret_cast<const TIO*>(args.f_base) + cell * n : nullptr;
  bool bad = false;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int x = 2 * mp + h;
    const TIO* fin = cell_input<TIO>(args, cell, x, n);
    const double vx = -L + x * dv, vz = -L + zp * dv;
    // Phi^T c at (vx, vy, vz) as a quadratic in the row index y: P0 + R(y)
    const double P0 = c5[0] + c5[1] * vx + c5[3] * vz + 0.5 * c5[4] * (vx * vx + vz * vz + L * L) - c5[2] * L;
    const uint32_t acol = accb + (uint32_t)(h * 32);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float a16[16];
      tmem_ld16(acol + 16 * c, a16);
      tmem_wait_ld16(a16);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int y = 16 * c + q;
        const int idx = (x * N + y) * N + zp;
        const TIO fv = fin[idx];
        double gv = gval(a16[q], fv);  // the same g as in the sums above
        if (fb) gv += args.a * to_f64(fb[idx]);
        const double val = gv + (P0 + Ry[y]);
        bad |= !isfinite(val);
        if (writable) out[idx] = from_f64<TIO>(val);
      }
    }
  }
  if (bad) atomicOr(&g_boltz_status, kStatusNonFinite);
  // every thread has read its last TMEM columns: free them
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(Cfg::TMEM_COLS));
}

// Launch: one CTA per cell, no term groups (a split launch needs clusters of the cell).
template <typename TIO>
static boltz_status launch_solo_impl(const CollideArgs& a, int64_t n_cells, cudaStream_t st) {
  using Cfg = SoloCfg;
  if (a.groups > 1) {
    set_error("the one-CTA-per-cell 32^3 kernel (cluster size 1) runs without term groups");
    return BOLTZ_EUNSUPPORTED;
  }
  auto kern = collide_solo_kernel<TIO>;
  static std::atomic<unsigned long long> prepared;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  const unsigned long long bit = 1ull << (dev & 63);
  size_t smem = Cfg::SMEM;
  const boltz_status ss = tmem_launch_smem(Cfg::TMEM_COLS, Cfg::SMEM, dev, &smem, 1);
  if (ss != BOLTZ_OK) return ss;
  if (dev >= 64 || !(prepared.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    if (dev < 64) prepared.fetch_or(bit, std::memory_order_release);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)n_cells, 1, 1);
  cfg.blockDim = dim3(Cfg::THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  e = cudaLaunchKernelEx(&cfg, kern, a);
  if (e != cudaSuccess) return cuda_fail(e, "collide launch");
  return BOLTZ_OK;
}

}  // namespace boltz
