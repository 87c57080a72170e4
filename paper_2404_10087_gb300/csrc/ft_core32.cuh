// Core-gradient pass, CTA-cooperative, FP32-accurate (K = 16 with N <= 5,
// K = 32 with N <= 4).
//
// The core gradient of Algorithm 5, G^(n) = sum_m (xhat_m - x_m) a^(n)_m^T d^(n)_m,
// as the BF16 cooperative pass computes it, with FP32-accurate arithmetic:
//   phase 1  each of the CTA's warps gathers its 16 nonzeros' float32 rows,
//            forms C^(n) = A_Psi B^(n) and xhat on three-pass TF32 products
//            (Prod<K, MATH_TF32X3>), D^(n) = *_{k != n} C^(k), and stages
//            A_Psi^(n) and (xhat - x) D^(n) as float32 rows in shared memory;
//   phase 2  the units (mode n, 16-row block mt of G^(n), one of H slices of
//            the CTA tile's nonzeros) are dealt to the warps, one each; a
//            unit contracts its slice, A_Psi^T ((xhat - x) D), into rows
//            16 mt .. 16 mt + 15 of G^(n) (all K columns) with three-pass
//            TF32 mma.sync m16n8k8 (operands split into TF32 head and tail,
//            lo.hi + hi.lo + hi.hi), and adds the slice's sums into
//            Neumaier-compensated registers once per CTA tile.
// At the end the slices of every block are combined in slice order into the
// CTA's partial ([n][K][K] of (sum, compensation) pairs, the layout
// k_finalize and k_batch_finalize reduce in fixed order), so the result is
// reproducible bit for bit.  The generic pass it replaces added compensated
// sums in shared memory for every 16 nonzeros.
#pragma once

#include "ft_device.cuh"

namespace ft {

template <int N, int K>
struct Core32 {
  static constexpr int CPL = K / 4;
  static constexpr int MT = K / 16;                            // 16-row blocks of G^(n)
  static constexpr int NT = K / 8;                             // 8-column n-tiles
  // K = 16: 4-warp CTAs (64-nonzero tiles, up to four per SM: shorter
  // barriers) up to N = 4, measured faster than 8-warp CTAs (9.2 against
  // 9.9 ms on the Netflix-shaped tensor); 8 warps at N = 5, where one unit
  // per mode needs them.  K = 32: 8 warps, one CTA per SM (registers).
  static constexpr int WARPS = (K == 16 && N <= 4) ? 4 : 8;
  static constexpr int ROWS = WARPS * FT_TILE;                 // nonzeros per CTA tile
  static constexpr int LD = K + 8;                             // floats per staged row: the
                                                               // fragment loads hit 32 banks
  static constexpr int BUF = ROWS * LD;                        // floats of one [ROWS][LD] buffer
  static constexpr int TW = Prod<K, MATH_TF32X3>::WORDS;       // a.B table per mode
  // slices of the CTA tile per block, so that the N * MT * H units keep most
  // warps busy in phase 2 (one unit per warp)
  static constexpr int H = (K == 32) ? 1 : (N == 1) ? 4 : (N == 2) ? 2 : 1;
  static constexpr int UNITS = N * MT * H;
  static constexpr int KSTEPS = ROWS / 8 / H;                  // k-steps of 8 nonzeros per unit
  static constexpr int ACC = 4 * NT;                           // accumulators per lane and unit
  static constexpr int MINB = (K == 16 && N <= 4) ? 4 : 1;     // CTAs per SM (K = 16: <= 128 registers)
  static constexpr size_t bytes() { return sizeof(float) * (size_t(N) * TW + size_t(2) * N * BUF); }
  static_assert(UNITS <= WARPS, "one unit per warp");
  static_assert((K == 16 && N <= 5) || (K == 32 && N <= 4), "other shapes take the generic pass");
  static_assert(UNITS * 2 * ACC * 32 <= 2 * N * BUF, "the combine's scratch fits in the row buffers");
};

// Phase 1 of one warp tile: stage A_Psi^(n) and (xhat - x) D^(n) of the warp's
// 16 nonzeros (rows 16 w .. 16 w + 15 of the CTA tile; masked nonzeros stage
// zero rows).
template <int N, int K>
__device__ __forceinline__ void core32_phase1(const EpochArgs &p, const TileCoords<N> &cur, const float *tabs,
                                              float *abuf, float *dbuf, int w, int lane) {
  using L = Core32<N, K>;
  constexpr int CPL = L::CPL;
  const int g = lane >> 2, t = lane & 3;
  Front<N, K, MATH_TF32X3, true> f;
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
      float *ad = abuf + n * L::BUF + row * L::LD + CPL * t;
      float *dd = dbuf + n * L::BUF + row * L::LD + CPL * t;
#pragma unroll
      for (int q = 0; q < CPL; q += 4) {
        *reinterpret_cast<float4 *>(ad + q) =
            make_float4(f.a[n][h][q], f.a[n][h][q + 1], f.a[n][h][q + 2], f.a[n][h][q + 3]);
        *reinterpret_cast<float4 *>(dd + q) = make_float4(ne[h] * d[h][q], ne[h] * d[h][q + 1],
                                                          ne[h] * d[h][q + 2], ne[h] * d[h][q + 3]);
      }
    }
  }
}

// Phase 2 of one unit (mode n, block mt, slice hh): the slice's contribution
// to rows 16 mt .. 16 mt + 15 of G^(n), accumulator element (u, i) at
// (j, r) = (16 mt + g + 8 (i / 2), 8 u + 2 t + i % 2); added into (gs, gc).
template <int N, int K>
__device__ __forceinline__ void core32_phase2(const float *abuf, const float *dbuf, int unit, int lane,
                                              float (&gs)[Core32<N, K>::ACC], float (&gc)[Core32<N, K>::ACC]) {
  using L = Core32<N, K>;
  constexpr int NT = L::NT;
  const int g = lane >> 2, t = lane & 3;
  const int n = unit / (L::MT * L::H), mt = (unit / L::H) % L::MT, hh = unit % L::H;
  const float *as = abuf + n * L::BUF + 16 * mt;
  const float *ds = dbuf + n * L::BUF;
  float acc[NT][4];
#pragma unroll
  for (int u = 0; u < NT; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.f;
#pragma unroll 4
  for (int kk = 0; kk < L::KSTEPS; ++kk) {
    const int m0 = 8 * (hh * L::KSTEPS + kk) + t, m1 = m0 + 4;
    // A operand A_Psi^T (rows j, contraction over the nonzeros m)
    uint32_t ah[4], al[4];
    Prod<K, MATH_TF32X3>::split(as[m0 * L::LD + g], ah[0], al[0]);
    Prod<K, MATH_TF32X3>::split(as[m0 * L::LD + g + 8], ah[1], al[1]);
    Prod<K, MATH_TF32X3>::split(as[m1 * L::LD + g], ah[2], al[2]);
    Prod<K, MATH_TF32X3>::split(as[m1 * L::LD + g + 8], ah[3], al[3]);
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      // B operand (xhat - x) D (contraction over m, columns r)
      uint32_t bh[2], bl[2];
      Prod<K, MATH_TF32X3>::split(ds[m0 * L::LD + 8 * u + g], bh[0], bl[0]);
      Prod<K, MATH_TF32X3>::split(ds[m1 * L::LD + 8 * u + g], bh[1], bl[1]);
      mma_tf32(acc[u], al[0], al[1], al[2], al[3], bh[0], bh[1]);
      mma_tf32(acc[u], ah[0], ah[1], ah[2], ah[3], bl[0], bl[1]);
      mma_tf32(acc[u], ah[0], ah[1], ah[2], ah[3], bh[0], bh[1]);
    }
  }
#pragma unroll
  for (int u = 0; u < NT; ++u)
#pragma unroll
    for (int i = 0; i < 4; ++i) neumaier_add(gs[4 * u + i], gc[4 * u + i], acc[u][i]);
}

// Combine the CTA's units into one partial at `out` ([n][K][K] of (sum,
// compensation) pairs): per element, the H slices of its block in slice
// order.  scratch: UNITS x 2 ACC x 32 floats of shared memory, free on entry
// (all warps past their last phase 2).  Ends with a barrier.
template <int N, int K>
__device__ __forceinline__ void core32_combine(float *scratch, int w, int lane, const float (&gs)[Core32<N, K>::ACC],
                                               const float (&gc)[Core32<N, K>::ACC], float *out) {
  using L = Core32<N, K>;
  constexpr int ACC = L::ACC;
  if (w < L::UNITS) {
#pragma unroll
    for (int q = 0; q < ACC; ++q) {
      scratch[(w * 2 * ACC + q) * 32 + lane] = gs[q];
      scratch[(w * 2 * ACC + ACC + q) * 32 + lane] = gc[q];
    }
  }
  __syncthreads();
  for (int f = threadIdx.x; f < N * K * K; f += blockDim.x) {
    const int n = f / (K * K), j = (f / K) % K, r = f % K;
    const int mt = j >> 4, jj = j & 15;
    const int g = jj & 7, ih = jj >> 3, u = r >> 3, t = (r & 7) >> 1, il = r & 1;
    const int q = 4 * u + 2 * ih + il, ln = 4 * g + t;
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int hh = 0; hh < L::H; ++hh) {
      const int unit = (n * L::MT + mt) * L::H + hh;
      neumaier_add(s, c, scratch[(unit * 2 * ACC + q) * 32 + ln]);
      c += scratch[(unit * 2 * ACC + ACC + q) * 32 + ln];
    }
    out[2 * f] = s;
    out[2 * f + 1] = c;
  }
  __syncthreads();
}

// Warp tiles [t_first + c * WARPS, ...) for CTA tiles c = c0, c0 + cs, ...
// below c_end, warp tiles clipped to t_end; (gs, gc) of the warp's unit.
template <int N, int K>
__device__ __forceinline__ void core32_tiles(const EpochArgs &p, const float *tabs, float *abuf, float *dbuf,
                                             int64_t t_first, int64_t t_end, int64_t c0, int64_t c_end,
                                             int64_t cs, float (&gs)[Core32<N, K>::ACC],
                                             float (&gc)[Core32<N, K>::ACC]) {
  using L = Core32<N, K>;
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
    core32_phase1<N, K>(p, cur, tabs, abuf, dbuf, w, lane);
    __syncthreads();
    if (w < L::UNITS) core32_phase2<N, K>(abuf, dbuf, w, lane, gs, gc);
    __syncthreads();
    cur = nxt;
  }
}

// Single tensor: CTA b takes CTA tiles b, b + G, ... of [begin, end) and
// writes its partial at p.partial + b * 2 N K K.
template <int N, int K>
__global__ void __launch_bounds__(32 * Core32<N, K>::WARPS, Core32<N, K>::MINB) k_core32(const EpochArgs p) {
  using L = Core32<N, K>;
  extern __shared__ __align__(16) float smem[];
  float *abuf = smem + N * L::TW;
  float *dbuf = abuf + N * L::BUF;
  fill_tables<N, K, MATH_TF32X3>(smem, p, false);
  float gs[L::ACC], gc[L::ACC];
#pragma unroll
  for (int q = 0; q < L::ACC; ++q) gs[q] = gc[q] = 0.f;
  __syncthreads();
  const int64_t ntiles = (p.end - p.begin + FT_TILE - 1) / FT_TILE;
  const int64_t nct = (ntiles + L::WARPS - 1) / L::WARPS;
  core32_tiles<N, K>(p, smem, abuf, dbuf, 0, ntiles, blockIdx.x, nct, gridDim.x, gs, gc);
  core32_combine<N, K>(abuf, threadIdx.x >> 5, threadIdx.x & 31, gs, gc,
                       p.partial + size_t(blockIdx.x) * 2 * N * K * K);
}

// Batched: the class's units (warp-tile ranges of one tensor each); CTA b
// takes units b, b + G, ...; every unit's partial goes to its own slot.
template <int N, int K>
__global__ void __launch_bounds__(32 * Core32<N, K>::WARPS, Core32<N, K>::MINB) k_batch_core32(const BatchArgs b) {
  using L = Core32<N, K>;
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
      fill_tables<N, K, MATH_TF32X3>(smem, ea, false);
      cur = un.tensor;
    }
    float gs[L::ACC], gc[L::ACC];
#pragma unroll
    for (int q = 0; q < L::ACC; ++q) gs[q] = gc[q] = 0.f;
    __syncthreads();
    const int64_t nct = (un.tile_end - un.tile_begin + L::WARPS - 1) / L::WARPS;
    core32_tiles<N, K>(ea, smem, abuf, dbuf, un.tile_begin, un.tile_end, 0, nct, 1, gs, gc);
    core32_combine<N, K>(abuf, threadIdx.x >> 5, threadIdx.x & 31, gs, gc, b.partial + un.poff);
  }
}

}  // namespace ft
