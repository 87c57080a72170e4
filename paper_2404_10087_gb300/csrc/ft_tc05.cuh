// Hogwild factor pass on the 5th-generation tensor cores (tcgen05 + TMEM),
// BF16 products with FP32 accumulation, padded rank K = 16, N <= 4.
//
// The same computation as k_factor (Algorithm 4 per sample set, Eq.
// "Update_FastTuckerPlus_factor" for the rows), re-tiled for sm_103a:
//   * a warpgroup owns a tile of 128 consecutive nonzeros - the M of one
//     tcgen05.mma - so C^(n) = A_Psi^(n) B^(n) and P^(n) = D^(n) B^(n)T are
//     one 128 x 16 x 16 MMA per mode, issued by one thread, with the
//     accumulators in tensor memory (TMEM) instead of registers;
//   * warp q of the warpgroup serves tile rows [32q, 32q + 32) (the TMEM
//     lanes it may access).  Lane 4g + t holds rows g + 8h (h = 0..3) of its
//     slab and columns [4t, 4t + 4): four lanes read one 64-byte factor row
//     (coalesced, as in the warp-tile kernel), and the 16x256b TMEM load
//     shape hands each lane exactly these rows and columns once the MMA's
//     N dimension (the B operand's rows) is permuted accordingly;
//   * the rows are staged for the MMA as BF16 in shared memory (canonical
//     K-major layout without swizzle), FP32 masters stay in registers for
//     the update; D^(n) reuses the same staging tiles.
// A CTA is 4 warpgroups (one persistent CTA per SM) sharing the operand
// tables of B and the hot-row write-back cache of k_factor.
#pragma once

#include "ft_device.cuh"

namespace ft {
namespace tc {

constexpr int TM = 128;                 // nonzeros per warpgroup tile (MMA M)
constexpr int WGS = 4;                  // warpgroups per CTA
constexpr int THREADS = 128 * WGS;
constexpr int OPND = TM * 16 * 2;       // bytes of one 128 x 16 BF16 operand tile
constexpr int BOPND = 16 * 16 * 2;      // bytes of one 16 x 16 BF16 operand
// Canonical K-major layout without swizzle: core matrices of 8 rows x 16
// bytes (row-major inside), LBO bytes between cores adjacent along K, SBO
// bytes between 8-row groups.
constexpr uint32_t LBO = 128, SBO = 256;
// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major, N = 16 (bits 17-22 = N / 8),
// M = 128 (bits 24-28 = M / 16).
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
// Polls of an mbarrier before a wait gives up (each poll may suspend briefly).
constexpr int SPIN = 1 << 22;

__device__ __forceinline__ uint32_t off_kmajor(int row, int k) {
  return uint32_t((row >> 3) * SBO + (k >> 3) * LBO + (row & 7) * 16 + (k & 7) * 2);
}

// Logical output column held by physical MMA column p: the 16x256b load gives
// lane 4g + t the physical columns {2t, 2t + 1, 8 + 2t, 9 + 2t}, which carry
// the logical columns 4t .. 4t + 3.
__device__ __forceinline__ int logical_col(int p) {
  return p < 8 ? 4 * (p >> 1) + (p & 1) : 4 * ((p - 8) >> 1) + 2 + (p & 1);
}

__device__ __forceinline__ uint32_t saddr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t(LBO >> 4) << 16) | (uint64_t(SBO >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(0));
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < SPIN && !done; ++it)
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  return done != 0;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void wg_sync(int wg) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + wg), "r"(128) : "memory");
}

// 16 lanes x 16 columns of TMEM: lane 4g + t gets rows g, g + 8 of the block
// in the order (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1), then the same for
// physical columns 8 + 2t, 9 + 2t.  The wait takes the registers as operands
// so that no use of them can move above it.
__device__ __forceinline__ void ld_block(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.16x256b.x2.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void ld_wait(uint32_t (&r)[8], uint32_t (&s)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3]), "+r"(s[4]), "+r"(s[5]), "+r"(s[6]), "+r"(s[7])
               :
               : "memory");
}

// The lane's 4 rows x 4 logical columns of one 16-column TMEM block pair
// (rows 0..15 and 16..31 of the warp's slab).
__device__ __forceinline__ void ld_rows(uint32_t taddr_slab, float (&v)[4][4]) {
  uint32_t r0[8], r1[8];
  ld_block(taddr_slab, r0);
  ld_block(taddr_slab + (16u << 16), r1);
  ld_wait(r0, r1);
#pragma unroll
  for (int hf = 0; hf < 2; ++hf) {
    const uint32_t(&r)[8] = hf ? r1 : r0;
    v[2 * hf][0] = __uint_as_float(r[0]);
    v[2 * hf][1] = __uint_as_float(r[1]);
    v[2 * hf][2] = __uint_as_float(r[4]);
    v[2 * hf][3] = __uint_as_float(r[5]);
    v[2 * hf + 1][0] = __uint_as_float(r[2]);
    v[2 * hf + 1][1] = __uint_as_float(r[3]);
    v[2 * hf + 1][2] = __uint_as_float(r[6]);
    v[2 * hf + 1][3] = __uint_as_float(r[7]);
  }
}

// Four BF16 values of one staged row (8 bytes).
__device__ __forceinline__ void st_op(unsigned char *tile, int row, int k0, const float (&v)[4]) {
  const uint32_t lo = pack_bf16(v[0], v[1]), hi = pack_bf16(v[2], v[3]);
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(saddr(tile + off_kmajor(row, k0))), "r"(lo), "r"(hi)
               : "memory");
}

template <int N>
struct Smem {
  static constexpr uint32_t BT = 0;                         // B operands of C = A B (rows: r, k: j)
  static constexpr uint32_t BN = BT + N * BOPND;            // B operands of P = D B^T (rows: j, k: r)
  static constexpr uint32_t OP = (BN + N * BOPND + 1023) / 1024 * 1024;  // [WGS][N] staging tiles
  static constexpr uint32_t BAR = OP + WGS * N * OPND;      // per warpgroup: MMA mbarrier, stage mbarrier
  static constexpr uint32_t TSLOT = BAR + 16 * WGS;         // TMEM base address
  static constexpr uint32_t HOT = (TSLOT + 16 + 15) / 16 * 16;  // hot-row cache, then dirty flags
  static constexpr uint32_t COLS_USED = WGS * 16 * N;
  static constexpr uint32_t TMEM_COLS = COLS_USED <= 32 ? 32 : COLS_USED <= 64 ? 64 : COLS_USED <= 128 ? 128 : 256;
  static constexpr size_t bytes(int hot_cap) {
    return HOT + size_t(hot_cap) * 16 * sizeof(float) + (size_t(hot_cap) + 15) / 16 * 16;
  }
  // the asynchronous row stage of one warpgroup: [N][TM] FP32 rows of 16
  static constexpr size_t STAGE_WG = size_t(N) * TM * 16 * sizeof(float);
  static constexpr size_t stage_bytes() { return WGS * STAGE_WG; }
};

// Coordinates and value of the lane's own slab row (loaded a tile ahead).
template <int N>
struct RowCoord {
  int32_t row[N];
  float x;
  bool valid;
  __device__ __forceinline__ void load(const EpochArgs &p, int64_t m) {
    valid = m < p.end;
#pragma unroll
    for (int n = 0; n < N; ++n) row[n] = valid ? __ldcs(p.idx[n] + m) : 0;
    x = valid ? __ldcs(p.vals + m) : 0.f;
  }
};

// One warpgroup tile.  Returns with every TMEM read of the tile done and
// fenced; `aborted` (warp-uniform) is set when an MMA completion wait gave up.
template <int N>
__device__ __forceinline__ void tile(const EpochArgs &p, unsigned char *sm, float *rep, unsigned char *dirty,
                                     const RowCoord<N> &rc, uint32_t tcol, uint32_t bar, uint32_t &phase,
                                     bool &aborted) {
  using L = Smem<N>;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int w = threadIdx.x >> 5, wg = w >> 2, q = w & 3;
  const bool issuer = (threadIdx.x & 127) == 0;
  unsigned char *op = sm + L::OP + uint32_t(wg * N) * OPND;
  const uint32_t tslab = tcol + (uint32_t(32 * q) << 16);

  // rows of this lane: slab row g + 8h, whose coordinates lane g + 8h loaded
  int32_t row[N][4];
  float x[4];
  bool valid[4];
  unsigned hot = 0u;
  bool bad = false;
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const int src = g + 8 * h;
    valid[h] = __shfl_sync(FULL, rc.valid, src);
    x[h] = __shfl_sync(FULL, rc.x, src);
    bool ok = true;
#pragma unroll
    for (int n = 0; n < N; ++n) {
      const int32_t v = __shfl_sync(FULL, rc.row[n], src);
      if (rep != nullptr && v < 0) {
        ok = ok && (-v - 1) >= p.hot_base[n] && (-v - 1) < p.hot_base[n + 1];
        row[n][h] = -v - 1;
        hot |= 1u << (4 * n + h);
      } else {
        ok = ok && v >= 0 && int64_t(v) < p.I[n];
        row[n][h] = v;
      }
    }
    if (valid[h] && !ok) {
      bad = true;
      valid[h] = false;
    }
    if (!valid[h]) {
      x[h] = 0.f;
#pragma unroll
      for (int n = 0; n < N; ++n) {
        row[n][h] = 0;
        hot &= ~(1u << (4 * n + h));
      }
    }
  }
  if (bad && t == 0) atomicOr(p.err, ERRBIT_INDEX);

  // gather the FP32 rows (a2) and stage them as BF16 (a3 operand of C = A B)
  float a[N][4][4];
#pragma unroll
  for (int n = 0; n < N; ++n) {
    const bool vec = ((p.vecmask >> n) & 1) != 0;
    const int Jn = p.J[n];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const bool is_hot = (hot >> (4 * n + h)) & 1u;
      const float *src = is_hot ? rep + size_t(row[n][h]) * 16 + 4 * t : p.A[n] + int64_t(row[n][h]) * Jn + 4 * t;
      float4 f4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid[h] && 4 * t < Jn) {
        if (vec || is_hot) {
          f4 = *reinterpret_cast<const float4 *>(src);
        } else {
          f4.x = src[0];
          if (4 * t + 1 < Jn) f4.y = src[1];
          if (4 * t + 2 < Jn) f4.z = src[2];
          if (4 * t + 3 < Jn) f4.w = src[3];
        }
      }
      a[n][h][0] = f4.x; a[n][h][1] = f4.y; a[n][h][2] = f4.z; a[n][h][3] = f4.w;
      st_op(op + n * OPND, 32 * q + g + 8 * h, 4 * t, a[n][h]);
    }
  }
  fence_async_smem();
  wg_sync(wg);
  if (issuer && !aborted) {
    fence_after();
#pragma unroll
    for (int n = 0; n < N; ++n)
      mma(tcol + 16 * n, sdesc(saddr(op + n * OPND)), sdesc(saddr(sm + L::BT + n * BOPND)));
    commit(bar);
  }
  {
    const bool ok = __all_sync(FULL, aborted ? false : wait_parity(bar, phase));
    phase ^= 1u;
    if (!ok && !aborted) {
      aborted = true;
      if (lane == 0) atomicOr(p.err, ERRBIT_TIMEOUT);
    }
  }
  fence_after();

  // prediction xhat = sum_r prod_n C^(n)_r and residual e (Eq. "fasttucker")
  float e[4];
  {
    float pr[4][4];
#pragma unroll
    for (int n = 0; n < N; ++n) {
      float c[4][4];
      if (!aborted) ld_rows(tslab + 16 * n, c);
      else {
#pragma unroll
        for (int h = 0; h < 4; ++h) c[h][0] = c[h][1] = c[h][2] = c[h][3] = 0.f;
      }
#pragma unroll
      for (int h = 0; h < 4; ++h)
#pragma unroll
        for (int k = 0; k < 4; ++k) pr[h][k] = n == 0 ? c[h][k] : pr[h][k] * c[h][k];
    }
    bool nf = false;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      float s = (pr[h][0] + pr[h][1]) + (pr[h][2] + pr[h][3]);
      s += __shfl_xor_sync(FULL, s, 1);
      s += __shfl_xor_sync(FULL, s, 2);
      e[h] = valid[h] ? x[h] - s : 0.f;
      nf = nf || (valid[h] && !isfinite(e[h]));
    }
    if (__any_sync(FULL, nf) && lane == 0) atomicOr(p.err, ERRBIT_NONFINITE);
  }

  // D^(n) = *_{k != n} C^(k) (Algorithm 4, Hadamard step), staged as the A
  // operand of P = D B^T in the tiles the rows occupied
#pragma unroll
  for (int n = 0; n < N; ++n) {
    float d[4][4];
#pragma unroll
    for (int h = 0; h < 4; ++h) d[h][0] = d[h][1] = d[h][2] = d[h][3] = 1.f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (k == n || aborted) continue;
      float c[4][4];
      ld_rows(tslab + 16 * k, c);
#pragma unroll
      for (int h = 0; h < 4; ++h)
#pragma unroll
        for (int j = 0; j < 4; ++j) d[h][j] *= c[h][j];
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) st_op(op + n * OPND, 32 * q + g + 8 * h, 4 * t, d[h]);
  }
  fence_async_smem();
  fence_before();
  wg_sync(wg);
  if (issuer && !aborted) {
    fence_after();
#pragma unroll
    for (int n = 0; n < N; ++n)
      mma(tcol + 16 * n, sdesc(saddr(op + n * OPND)), sdesc(saddr(sm + L::BN + n * BOPND)));
    commit(bar);
  }
  {
    const bool ok = __all_sync(FULL, aborted ? false : wait_parity(bar, phase));
    phase ^= 1u;
    if (!ok && !aborted) {
      aborted = true;
      if (lane == 0) atomicOr(p.err, ERRBIT_TIMEOUT);
    }
  }
  fence_after();

  // a <- a + lr * s_row * (e P - lam a), stored to the cache or to global memory
#pragma unroll
  for (int n = 0; n < N; ++n) {
    float pp[4][4];
    if (aborted) break;
    ld_rows(tslab + 16 * n, pp);
    const bool vec = ((p.vecmask >> n) & 1) != 0;
    const int Jn = p.J[n];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      if (!valid[h] || 4 * t >= Jn) continue;
      const bool is_hot = (hot >> (4 * n + h)) & 1u;
      float lr = p.lr;
      if (p.scale[n]) {
        const int64_t grow = is_hot ? int64_t(__ldg(p.hot_rows + row[n][h])) : int64_t(row[n][h]);
        lr *= __ldg(p.scale[n] + grow);
      }
      float o[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) o[j] = fmaf(lr, fmaf(e[h], pp[h][j], -p.lam * a[n][h][j]), a[n][h][j]);
      float *dst = is_hot ? rep + size_t(row[n][h]) * 16 + 4 * t : p.A[n] + int64_t(row[n][h]) * Jn + 4 * t;
      if (vec || is_hot) {
        *reinterpret_cast<float4 *>(dst) = make_float4(o[0], o[1], o[2], o[3]);
      } else {
        dst[0] = o[0];
        if (4 * t + 1 < Jn) dst[1] = o[1];
        if (4 * t + 2 < Jn) dst[2] = o[2];
        if (4 * t + 3 < Jn) dst[3] = o[3];
      }
      if (is_hot && t == 0) dirty[row[n][h]] = 1;
    }
  }
  fence_before();
}

// ---------------------------------------------------- asynchronous row stage
// The tile's rows as the thread that owns the tile row sees them (thread
// 32 q + lane of a warpgroup owns row 32 q + lane): per mode the global row or
// cache slot and whether it is hot, the value and whether the nonzero is
// valid (inside the range, every coordinate in bounds).
template <int N>
struct RowDec {
  uint32_t r[N];
  unsigned hot;        // bit n
  bool valid;
  float x;
  // returns true when a valid nonzero had a coordinate out of bounds
  __device__ __forceinline__ bool decode(const EpochArgs &p, const RowCoord<N> &rc) {
    bool ok = true;
    hot = 0u;
#pragma unroll
    for (int n = 0; n < N; ++n) {
      const int32_t v = rc.row[n];
      const bool is_hot = v < 0;
      const uint32_t slot = ~uint32_t(v);
      ok = ok && (is_hot ? slot - uint32_t(p.hot_base[n]) < uint32_t(p.hot_base[n + 1] - p.hot_base[n])
                         : uint32_t(v) < uint32_t(p.I[n]));
      r[n] = is_hot ? slot : uint32_t(v);
      hot |= unsigned(is_hot) << n;
    }
    const bool bad = rc.valid && !ok;
    valid = rc.valid && ok;
    x = valid ? rc.x : 0.f;
    if (!valid) {
      hot = 0u;
#pragma unroll
      for (int n = 0; n < N; ++n) r[n] = 0u;
    }
    return bad;
  }
};

// The warp copies the cold rows of its 32 tile rows (owned by its lanes)
// into the stage: lane 4 g + t copies the 16-byte quarter t of rows g + 8 h,
// h = 0..3, of every mode with cp.async (the fast path's rows are full width,
// 64 bytes, 16-byte aligned), so each copy instruction of the warp moves eight
// whole rows.  Each thread then arrives on the warpgroup's stage mbarrier
// (count 128) once its own copies have landed (arrive.noinc), so the phase
// completes when every copy of the warpgroup has.  Hot and invalid rows copy
// nothing; a thread without copies arrives at once.
template <int N>
__device__ __forceinline__ void stage_issue(const EpochArgs &p, const RowDec<N> &d, unsigned char *stage, int q,
                                            int lane, uint32_t bar) {
  const int g = lane >> 2, t = lane & 3;
  const unsigned cold = d.valid ? (~d.hot & ((1u << N) - 1u)) : 0u;
  const uint32_t base = saddr(stage) + uint32_t((32 * q + g) * 64 + 16 * t);
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const unsigned cb = __shfl_sync(FULL, cold, g + 8 * h);
#pragma unroll
    for (int n = 0; n < N; ++n) {
      const uint32_t rn = __shfl_sync(FULL, d.r[n], g + 8 * h);
      const float *src = p.A[n] + size_t(rn) * 16 + 4 * t;
      const uint32_t dst = base + uint32_t((n * TM + 8 * h) * 64);
      asm volatile(
          "{\n\t.reg .pred pc;\n\tsetp.ne.b32 pc, %2, 0;\n\t"
          "@pc cp.async.cg.shared.global [%0], [%1], 16;\n\t}" ::"r"(dst),
          "l"(src), "r"((cb >> n) & 1u)
          : "memory");
    }
  }
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// One warpgroup tile with its cold rows arriving in the stage (started one
// tile ahead by stage_issue) and hot rows read from the cache: the same
// arithmetic as tile(), written without data-dependent branches.  After the
// rows have been read (and the warpgroup has synchronised) the owners of the
// next tile's rows start its copies, so they overlap this tile's products.
// `active`: this warpgroup has a tile here (otherwise only the stage
// protocol runs).  Returns with every TMEM read of the tile done and fenced.
template <int N>
__device__ __forceinline__ void tile_async(const EpochArgs &p, unsigned char *sm, float *rep, unsigned char *dirty,
                                           unsigned char *stage, const RowDec<N> &own, bool active,
                                           bool has_next, RowDec<N> &own_next, const RowCoord<N> &next_rc,
                                           uint32_t tcol, uint32_t bar, uint32_t sbar, uint32_t &phase,
                                           uint32_t &sphase, bool &aborted) {
  using L = Smem<N>;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int w = threadIdx.x >> 5, wg = w >> 2, q = w & 3;
  const bool issuer = (threadIdx.x & 127) == 0;
  unsigned char *op = sm + L::OP + uint32_t(wg * N) * OPND;
  const uint32_t tslab = tcol + (uint32_t(32 * q) << 16);
  const uint32_t rep_s = saddr(rep != nullptr ? rep : reinterpret_cast<float *>(sm));
  const uint32_t stage_s = saddr(stage);

  // this tile's rows have arrived
  {
    const bool ok = __all_sync(FULL, aborted ? false : wait_parity(sbar, sphase));
    sphase ^= 1u;
    if (!ok && !aborted) {
      aborted = true;
      if (lane == 0) atomicOr(p.err, ERRBIT_TIMEOUT);
    }
  }
  // the lane's rows g + 8h of its slab, from the owners g + 8h
  uint32_t r[N][4];
  unsigned hot = 0u;
  float x[4];
  bool valid[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const int src = g + 8 * h;
    valid[h] = __shfl_sync(FULL, own.valid, src);
    x[h] = __shfl_sync(FULL, own.x, src);
    const unsigned hb = __shfl_sync(FULL, own.hot, src);
#pragma unroll
    for (int n = 0; n < N; ++n) {
      r[n][h] = __shfl_sync(FULL, own.r[n], src);
      hot |= ((hb >> n) & 1u) << (4 * n + h);
    }
  }
  // gather (a2) and stage as the BF16 operand of C = A B (a3)
  float a[N][4][4];
#pragma unroll
  for (int n = 0; n < N; ++n)
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const bool is_hot = (hot >> (4 * n + h)) & 1u;
      const uint32_t src = is_hot ? rep_s + (r[n][h] * 16 + 4 * t) * 4u
                                  : stage_s + uint32_t((n * TM + 32 * q + g + 8 * h) * 16 + 4 * t) * 4u;
      float4 f4;
      asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(f4.x), "=f"(f4.y), "=f"(f4.z), "=f"(f4.w) : "r"(src)
                   : "memory");
      a[n][h][0] = valid[h] ? f4.x : 0.f;
      a[n][h][1] = valid[h] ? f4.y : 0.f;
      a[n][h][2] = valid[h] ? f4.z : 0.f;
      a[n][h][3] = valid[h] ? f4.w : 0.f;
      st_op(op + n * OPND, 32 * q + g + 8 * h, 4 * t, a[n][h]);
    }
  fence_async_smem();
  wg_sync(wg);
  // every thread of the warpgroup has read the stage: start the next tile's
  // copies (after a timeout only the arrival, so the phase still completes)
  if (has_next) {
    const bool bad = own_next.decode(p, next_rc);
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(p.err, ERRBIT_INDEX);
    if (aborted) own_next.valid = false;
    stage_issue<N>(p, own_next, stage, q, lane, sbar);
  }
  if (!active) return;
  if (issuer && !aborted) {
    fence_after();
#pragma unroll
    for (int n = 0; n < N; ++n)
      mma(tcol + 16 * n, sdesc(saddr(op + n * OPND)), sdesc(saddr(sm + L::BT + n * BOPND)));
    commit(bar);
  }
  {
    const bool ok = __all_sync(FULL, aborted ? false : wait_parity(bar, phase));
    phase ^= 1u;
    if (!ok && !aborted) {
      aborted = true;
      if (lane == 0) atomicOr(p.err, ERRBIT_TIMEOUT);
    }
  }
  fence_after();

  // prediction and residual (Eq. "fasttucker")
  float e[4];
  {
    float pr[4][4];
#pragma unroll
    for (int n = 0; n < N; ++n) {
      float c[4][4];
      if (!aborted) ld_rows(tslab + 16 * n, c);
      else {
#pragma unroll
        for (int h = 0; h < 4; ++h) c[h][0] = c[h][1] = c[h][2] = c[h][3] = 0.f;
      }
#pragma unroll
      for (int h = 0; h < 4; ++h)
#pragma unroll
        for (int k = 0; k < 4; ++k) pr[h][k] = n == 0 ? c[h][k] : pr[h][k] * c[h][k];
    }
    bool nf = false;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      float s = (pr[h][0] + pr[h][1]) + (pr[h][2] + pr[h][3]);
      s += __shfl_xor_sync(FULL, s, 1);
      s += __shfl_xor_sync(FULL, s, 2);
      e[h] = valid[h] ? x[h] - s : 0.f;
      nf = nf || (valid[h] && !isfinite(e[h]));
    }
    if (__any_sync(FULL, nf) && lane == 0) atomicOr(p.err, ERRBIT_NONFINITE);
  }

  // D^(n) = *_{k != n} C^(k), staged as the A operand of P = D B^T
#pragma unroll
  for (int n = 0; n < N; ++n) {
    float d[4][4];
#pragma unroll
    for (int h = 0; h < 4; ++h) d[h][0] = d[h][1] = d[h][2] = d[h][3] = 1.f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (k == n || aborted) continue;
      float c[4][4];
      ld_rows(tslab + 16 * k, c);
#pragma unroll
      for (int h = 0; h < 4; ++h)
#pragma unroll
        for (int j = 0; j < 4; ++j) d[h][j] *= c[h][j];
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) st_op(op + n * OPND, 32 * q + g + 8 * h, 4 * t, d[h]);
  }
  fence_async_smem();
  fence_before();
  wg_sync(wg);
  if (issuer && !aborted) {
    fence_after();
#pragma unroll
    for (int n = 0; n < N; ++n)
      mma(tcol + 16 * n, sdesc(saddr(op + n * OPND)), sdesc(saddr(sm + L::BN + n * BOPND)));
    commit(bar);
  }
  {
    const bool ok = __all_sync(FULL, aborted ? false : wait_parity(bar, phase));
    phase ^= 1u;
    if (!ok && !aborted) {
      aborted = true;
      if (lane == 0) atomicOr(p.err, ERRBIT_TIMEOUT);
    }
  }
  fence_after();

  // a <- (1 - lr lam) a + (lr e) P, to the cache or to global memory (the
  // BF16 products' rounding dwarfs the row's float32 roundings)
  const float keep = 1.f - p.lr * p.lam;
#pragma unroll
  for (int n = 0; n < N; ++n) {
    float pp[4][4];
    if (aborted) break;
    ld_rows(tslab + 16 * n, pp);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const bool is_hot = (hot >> (4 * n + h)) & 1u;
      const float ge = p.lr * e[h];
      float *dst = is_hot ? rep + size_t(r[n][h]) * 16 + 4 * t : p.A[n] + size_t(r[n][h]) * 16 + 4 * t;
      const float4 o = make_float4(fmaf(ge, pp[h][0], keep * a[n][h][0]), fmaf(ge, pp[h][1], keep * a[n][h][1]),
                                   fmaf(ge, pp[h][2], keep * a[n][h][2]), fmaf(ge, pp[h][3], keep * a[n][h][3]));
      if (valid[h]) *reinterpret_cast<float4 *>(dst) = o;
      if (valid[h] && is_hot && t == 0) dirty[r[n][h]] = 1;
    }
  }
  fence_before();
}

}  // namespace tc

// One Hogwild pass of the factor update over [begin, end) on tcgen05.
// Warpgroup wg of CTA b takes the 128-nonzero tiles 4c + wg for c = b, b + G,
// ...  With the hot-row cache on, the CTA writes its dirty rows back and
// refreshes them every max(1, hot_window / 4) CTA tiles, i.e. after the same
// number of nonzeros per CTA as k_factor.  A timed-out MMA wait latches
// ERRBIT_TIMEOUT; the CTA stops at its next window boundary and frees TMEM.
// ASYNC (hot-row cache on, every row full width, one step size): the rows
// of the next tile arrive in a per-warpgroup stage by asynchronous copies
// (stage_issue, tile_async).
template <int N, bool ASYNC = false>
__global__ void __launch_bounds__(tc::THREADS, 1) k_factor_tc(const EpochArgs p) {
  using L = tc::Smem<N>;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, w = tid >> 5, wg = w >> 2, q = w & 3, lane = tid & 31;

  // operand tables of B^(n) (BF16, zero padded, MMA N dimension permuted)
  for (int e = tid; e < N * 256; e += tc::THREADS) {
    const int n = e >> 8, pr = (e >> 4) & 15, k = e & 15;
    const int l = tc::logical_col(pr);
    const float vt = (k < p.J[n] && l < p.R) ? __ldg(p.B[n] + k * p.R + l) : 0.f;
    const float vn = (l < p.J[n] && k < p.R) ? __ldg(p.B[n] + l * p.R + k) : 0.f;
    *reinterpret_cast<__nv_bfloat16 *>(sm + L::BT + n * tc::BOPND + tc::off_kmajor(pr, k)) = __float2bfloat16_rn(vt);
    *reinterpret_cast<__nv_bfloat16 *>(sm + L::BN + n * tc::BOPND + tc::off_kmajor(pr, k)) = __float2bfloat16_rn(vn);
  }
  const bool cache = p.hot_cap > 0;
  float *rep = cache ? reinterpret_cast<float *>(sm + L::HOT) : nullptr;
  unsigned char *dirty = cache ? sm + L::HOT + size_t(p.hot_cap) * 16 * sizeof(float) : nullptr;
  if (cache) {
    cache_refresh<N, 16>(p, rep);
    for (int e = tid; e < p.hot_cap; e += tc::THREADS) dirty[e] = 0;
  }
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L::BAR);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + L::TSLOT);
  if (tid == 0) {
    for (int b = 0; b < tc::WGS; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::saddr(bars + b)), "r"(1) : "memory");
      // stage barrier: every thread of the warpgroup arrives once per tile
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::saddr(bars + tc::WGS + b)), "r"(128)
                   : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::saddr(tslot)),
                 "r"(L::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t tcol = tbase + uint32_t(wg * 16 * N);
  const uint32_t bar = tc::saddr(bars + wg);
  uint32_t phase = 0;
  bool aborted = false;

  const int64_t ntiles = (p.end - p.begin + tc::TM - 1) / tc::TM;
  const int64_t nct = (ntiles + tc::WGS - 1) / tc::WGS;
  const int64_t G = gridDim.x;
  const int W = (cache && p.hot_window > 0) ? (p.hot_window + tc::WGS - 1) / tc::WGS : 16;
  if constexpr (ASYNC) {
    // the warpgroup's stage follows the dirty flags
    unsigned char *stage = dirty + (size_t(p.hot_cap) + 15) / 16 * 16 + size_t(wg) * L::STAGE_WG;
    const uint32_t sbar = tc::saddr(bars + tc::WGS + wg);
    uint32_t sphase = 0;
    auto row_of = [&](int64_t c) { return p.begin + (c * tc::WGS + wg) * tc::TM + 32 * q + lane; };
    tc::RowCoord<N> rc;
    tc::RowDec<N> d0, d1;
    if (blockIdx.x < nct) {
      rc.load(p, row_of(blockIdx.x));
      const bool bad = d0.decode(p, rc);
      if (__any_sync(FULL, bad) && lane == 0) atomicOr(p.err, ERRBIT_INDEX);
      tc::stage_issue<N>(p, d0, stage, q, lane, sbar);
    }
    if (blockIdx.x + G < nct) rc.load(p, row_of(blockIdx.x + G));
    int k = 0;
    bool pending = blockIdx.x < nct;   // a stage phase was started and not waited for
    auto step = [&](int64_t c, const tc::RowDec<N> &cur, tc::RowDec<N> &nxt) -> bool {
      const int64_t c1 = c + G, c2 = c + 2 * G;
      tc::tile_async<N>(p, sm, rep, dirty, stage, cur, c * tc::WGS + wg < ntiles, c1 < nct, nxt, rc, tcol, bar,
                        sbar, phase, sphase, aborted);
      pending = c1 < nct;
      if (c2 < nct) rc.load(p, row_of(c2));
      if (++k == W || c1 >= nct) {
        k = 0;
        const bool stop = __syncthreads_or(aborted) != 0;
        cache_write_back<N, 16>(p, rep, dirty);
        if (stop) return false;
        if (c1 < nct) {
          __syncthreads();
          cache_refresh<N, 16>(p, rep);
          __syncthreads();
        }
      }
      return c1 < nct;
    };
    for (int64_t c = blockIdx.x; c < nct; c += 2 * G) {
      if (!step(c, d0, d1)) break;
      if (!step(c + G, d1, d0)) break;
    }
    // copies started for a tile that never ran (a stop after a timeout):
    // wait for them, with a limit, before the CTA leaves
    if (pending) (void)tc::wait_parity(sbar, sphase);
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else {
  tc::RowCoord<N> cur, nxt;
  if (blockIdx.x < nct) cur.load(p, p.begin + (int64_t(blockIdx.x) * tc::WGS + wg) * tc::TM + 32 * q + lane);
  int k = 0;
  for (int64_t c = blockIdx.x; c < nct; c += G) {
    const int64_t cn = c + G;
    if (cn < nct) nxt.load(p, p.begin + (cn * tc::WGS + wg) * tc::TM + 32 * q + lane);
    if (c * tc::WGS + wg < ntiles) tc::tile<N>(p, sm, rep, dirty, cur, tcol, bar, phase, aborted);
    cur = nxt;
    if (++k == W || cn >= nct) {
      k = 0;
      const bool stop = __syncthreads_or(aborted) != 0;
      if (cache) cache_write_back<N, 16>(p, rep, dirty);
      if (stop) break;
      if (cache && cn < nct) {
        __syncthreads();
        cache_refresh<N, 16>(p, rep);
        __syncthreads();
      }
    }
  }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (w == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(L::TMEM_COLS) : "memory");
}

}  // namespace ft
