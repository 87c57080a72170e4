// Core-gradient pass, CTA-cooperative, FP32-accurate (K = 16, N <= 5).
//
// The core gradient of Algorithm 5, G^(n) = sum_m (xhat_m - x_m) a^(n)_m^T d^(n)_m,
// as the BF16 cooperative pass computes it, with FP32-accurate arithmetic:
//   phase 1  each of the CTA's warps gathers its 16 nonzeros' float32 rows,
//            forms C^(n) = A_Psi B^(n) and xhat on three-pass TF32 products
//            (Prod<16, MATH_TF32X3>), D^(n) = *_{k != n} C^(k), and stages
//            A_Psi^(n) and (xhat - x) D^(n) as float32 rows in shared memory;
//   phase 2  the N x H units (mode n, one of H slices of the CTA tile's 64
//            or 128 nonzeros) are dealt to the warps; each contracts its slice,
//            A_Psi^T ((xhat - x) D), into the 16 x 16 block of G^(n) with
//            three-pass TF32 mma.sync m16n8k8 (operands split into TF32 head
//            and tail, lo.hi + hi.lo + hi.hi), and adds the slice's sums into
//            Neumaier-compensated registers once per CTA tile.
// At the end the units of a mode are combined in slice order into the CTA's
// partial ([n][K][K] of (sum, compensation) pairs, the layout k_finalize and
// k_batch_finalize reduce in fixed order), so the result is reproducible bit
// for bit.  The generic pass it replaces added compensated sums in shared
// memory for every 16 nonzeros.
#pragma once

#include "ft_device.cuh"

namespace ft {

template <int N>
struct Core32 {
  static constexpr int K = 16;
  static constexpr int CPL = K / 4;
  // 4-warp CTAs (64-nonzero tiles, up to four per SM: shorter barriers) up to
  // N = 4, measured faster than 8-warp CTAs (9.2 against 9.9 ms on the
  // Netflix-shaped tensor); 8 warps at N = 5, where one unit per mode needs them
  static constexpr int WARPS = (N <= 4) ? 4 : 8;
  static constexpr int ROWS = WARPS * FT_TILE;                 // nonzeros per CTA tile
  static constexpr int LD = K + 8;                             // floats per staged row: the
                                                               // fragment loads hit 32 banks
  static constexpr int BUF = ROWS * LD;                        // floats of one [ROWS][LD] buffer
  static constexpr int TW = Prod<K, MATH_TF32X3>::WORDS;       // a.B table per mode
  // slices of the CTA tile per mode, so that the N * H units keep most
  // warps busy in phase 2 (N * H <= WARPS)
  static constexpr int H = (N == 1) ? 4 : (N == 2) ? 2 : 1;
  static constexpr int UNITS = N * H;
  static constexpr int KSTEPS = ROWS / 8 / H;                  // k-steps of 8 nonzeros per unit
  static constexpr int MINB = (N <= 4) ? 4 : 1;                // CTAs per SM (registers <= 128)
  static constexpr size_t bytes() { return sizeof(float) * (size_t(N) * TW + size_t(2) * N * BUF); }
  static_assert(UNITS <= WARPS, "one unit per warp");
  static_assert(N <= 5, "orders above 5 take the generic pass");
};

// Phase 1 of one warp tile: stage A_Psi^(n) and (xhat - x) D^(n) of the warp's
// 16 nonzeros (rows 16 w .. 16 w + 15 of the CTA tile; masked nonzeros stage
// zero rows).
template <int N>
__device__ __forceinline__ void core32_phase1(const EpochArgs &p, const TileCoords<N> &cur, const float *tabs,
                                              float *abuf, float *dbuf, int w, int lane) {
  using L = Core32<N>;
  constexpr int CPL = L::CPL;
  const int g = lane >> 2, t = lane & 3;
  Front<N, L::K, MATH_TF32X3, true> f;
  f.gather(p, cur, lane);
  f.compute(tabs, L::TW, lane);
  float ne[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) ne[h] = f.valid[h] ? f.xhat[h] - f.x[h] : 0.f;
  const bool nonfinite = !isfinite(ne[0]) || !isfinite(ne[1]);
  if (__any_sync(FULL, nonfinite) && lane == 0) atomicOr(p.err, ERRBIT_NONFINITE);
#pragma unroll
  for (int n = 0; n < N; ++n) {
    float d[2][CPL];
    f.leave_one_out(n, d);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = FT_TILE * w + g + 8 * h;
      *reinterpret_cast<float4 *>(abuf + n * L::BUF + row * L::LD + CPL * t) =
          make_float4(f.a[n][h][0], f.a[n][h][1], f.a[n][h][2], f.a[n][h][3]);
      *reinterpret_cast<float4 *>(dbuf + n * L::BUF + row * L::LD + CPL * t) =
          make_float4(ne[h] * d[h][0], ne[h] * d[h][1], ne[h] * d[h][2], ne[h] * d[h][3]);
    }
  }
}

// Phase 2 of one unit (mode n, slice hh): the slice's contribution to the
// 16 x 16 block of G^(n), accumulator element (u, i) at
// (j, r) = (g + 8 (i / 2), 8 u + 2 t + i % 2); added into (gs, gc).
template <int N>
__device__ __forceinline__ void core32_phase2(const float *abuf, const float *dbuf, int unit, int lane,
                                              float (&gs)[8], float (&gc)[8]) {
  using L = Core32<N>;
  const int g = lane >> 2, t = lane & 3;
  const int n = unit / L::H, hh = unit % L::H;
  const float *as = abuf + n * L::BUF;
  const float *ds = dbuf + n * L::BUF;
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll 4
  for (int kk = 0; kk < L::KSTEPS; ++kk) {
    const int m0 = 8 * (hh * L::KSTEPS + kk) + t, m1 = m0 + 4;
    // A operand A_Psi^T (rows j, contraction over the nonzeros m)
    uint32_t ah[4], al[4];
    Prod<16, MATH_TF32X3>::split(as[m0 * L::LD + g], ah[0], al[0]);
    Prod<16, MATH_TF32X3>::split(as[m0 * L::LD + g + 8], ah[1], al[1]);
    Prod<16, MATH_TF32X3>::split(as[m1 * L::LD + g], ah[2], al[2]);
    Prod<16, MATH_TF32X3>::split(as[m1 * L::LD + g + 8], ah[3], al[3]);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      // B operand (xhat - x) D (contraction over m, columns r)
      uint32_t bh[2], bl[2];
      Prod<16, MATH_TF32X3>::split(ds[m0 * L::LD + 8 * u + g], bh[0], bl[0]);
      Prod<16, MATH_TF32X3>::split(ds[m1 * L::LD + 8 * u + g], bh[1], bl[1]);
      mma_tf32(acc[u], al[0], al[1], al[2], al[3], bh[0], bh[1]);
      mma_tf32(acc[u], ah[0], ah[1], ah[2], ah[3], bl[0], bl[1]);
      mma_tf32(acc[u], ah[0], ah[1], ah[2], ah[3], bh[0], bh[1]);
    }
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int i = 0; i < 4; ++i) neumaier_add(gs[4 * u + i], gc[4 * u + i], acc[u][i]);
}

// Combine the CTA's units into one partial at `out` ([n][16][16] of (sum,
// compensation) pairs): per element, the H slices of its mode in slice order.
// scratch: UNITS x 16 x 32 floats of shared memory, free on entry (all
// warps past their last phase 2).  Ends with a barrier.
template <int N>
__device__ __forceinline__ void core32_combine(float *scratch, int w, int lane, const float (&gs)[8],
                                               const float (&gc)[8], float *out) {
  using L = Core32<N>;
  if (w < L::UNITS) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      scratch[(w * 16 + q) * 32 + lane] = gs[q];
      scratch[(w * 16 + 8 + q) * 32 + lane] = gc[q];
    }
  }
  __syncthreads();
  for (int f = threadIdx.x; f < N * 256; f += blockDim.x) {
    const int n = f >> 8, j = (f >> 4) & 15, r = f & 15;
    const int g = j & 7, ih = j >> 3, u = r >> 3, t = (r & 7) >> 1, il = r & 1;
    const int q = 4 * u + 2 * ih + il, ln = 4 * g + t;
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int hh = 0; hh < L::H; ++hh) {
      const int unit = n * L::H + hh;
      neumaier_add(s, c, scratch[(unit * 16 + q) * 32 + ln]);
      c += scratch[(unit * 16 + 8 + q) * 32 + ln];
    }
    out[2 * f] = s;
    out[2 * f + 1] = c;
  }
  __syncthreads();
}

// Warp tiles [t_first + c * WARPS, ...) for CTA tiles c = c0, c0 + cs, ...
// below c_end, warp tiles clipped to t_end; (gs, gc) of the warp's unit.
template <int N>
__device__ __forceinline__ void core32_tiles(const EpochArgs &p, const float *tabs, float *abuf, float *dbuf,
                                             int64_t t_first, int64_t t_end, int64_t c0, int64_t c_end,
                                             int64_t cs, float (&gs)[8], float (&gc)[8]) {
  using L = Core32<N>;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // a warp tile past t_end loads no nonzeros (its coordinates start at p.end)
  auto base = [&](int64_t c) {
    const int64_t tile = t_first + c * L::WARPS + w;
    return tile < t_end ? p.begin + tile * FT_TILE : p.end;
  };
  TileCoords<N> cur, nxt;
  if (c0 < c_end) cur.load(p, base(c0), lane, true);
  for (int64_t c = c0; c < c_end; c += cs) {
    const int64_t cn = c + cs;
    if (cn < c_end) nxt.load(p, base(cn), lane, true);
    core32_phase1<N>(p, cur, tabs, abuf, dbuf, w, lane);
    __syncthreads();
    if (w < L::UNITS) core32_phase2<N>(abuf, dbuf, w, lane, gs, gc);
    __syncthreads();
    cur = nxt;
  }
}

// Single tensor: CTA b takes CTA tiles b, b + G, ... of [begin, end) and
// writes its partial at p.partial + b * 2 N K K.
template <int N>
__global__ void __launch_bounds__(32 * Core32<N>::WARPS, Core32<N>::MINB) k_core32(const EpochArgs p) {
  using L = Core32<N>;
  extern __shared__ __align__(16) float smem[];
  float *abuf = smem + N * L::TW;
  float *dbuf = abuf + N * L::BUF;
  fill_tables<N, L::K, MATH_TF32X3>(smem, p, false);
  float gs[8], gc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) gs[q] = gc[q] = 0.f;
  __syncthreads();
  const int64_t ntiles = (p.end - p.begin + FT_TILE - 1) / FT_TILE;
  const int64_t nct = (ntiles + L::WARPS - 1) / L::WARPS;
  core32_tiles<N>(p, smem, abuf, dbuf, 0, ntiles, blockIdx.x, nct, gridDim.x, gs, gc);
  core32_combine<N>(abuf, threadIdx.x >> 5, threadIdx.x & 31, gs, gc,
                    p.partial + size_t(blockIdx.x) * 2 * N * L::K * L::K);
}

// Batched: the class's units (warp-tile ranges of one tensor each); CTA b
// takes units b, b + G, ...; every unit's partial goes to its own slot.
template <int N>
__global__ void __launch_bounds__(32 * Core32<N>::WARPS, Core32<N>::MINB) k_batch_core32(const BatchArgs b) {
  using L = Core32<N>;
  extern __shared__ __align__(16) float smem[];
  __shared__ EpochArgs ea;
  float *abuf = smem + N * L::TW;
  float *dbuf = abuf + N * L::BUF;
  int cur = -1;
  for (int u = blockIdx.x; u < b.nunits; u += gridDim.x) {
    const BatchUnit un = b.units[u];
    if (un.tensor != cur) {
      if (threadIdx.x == 0) ea = b.tensors[un.tensor];
      __syncthreads();
      fill_tables<N, L::K, MATH_TF32X3>(smem, ea, false);
      cur = un.tensor;
    }
    float gs[8], gc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) gs[q] = gc[q] = 0.f;
    __syncthreads();
    const int64_t nct = (un.tile_end - un.tile_begin + L::WARPS - 1) / L::WARPS;
    core32_tiles<N>(ea, smem, abuf, dbuf, un.tile_begin, un.tile_end, 0, nct, 1, gs, gc);
    core32_combine<N>(abuf, threadIdx.x >> 5, threadIdx.x & 31, gs, gc, b.partial + un.poff);
  }
}

}  // namespace ft
