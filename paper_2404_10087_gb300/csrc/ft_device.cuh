// Device side of the FastTuckerPlus epoch for sm_103a.
//
// Work decomposition (Sec. 4.3-4.4 of the paper: one warp per sample set Psi
// of M = 16 nonzeros, grid-stride over the Psi): a warp owns a tile of 16
// consecutive nonzeros.  Lane l = 4g + t (g = l / 4 in 0..7, t = l % 4 in
// 0..3) holds tile rows g and g + 8, and in each of them the column chunk
// [CPL*t, CPL*t + CPL) with CPL = K / 4, K the padded rank (16 or 32).
// This "row-chunk" layout is shared by A_Psi (columns j), C_Psi and D_Psi
// (columns r) and P = D B^T (columns j):
//   * a chunk of a factor row is one 16-byte vector load per 4 columns;
//   * the tensor-core products are arranged (by permuting the contraction
//     index and the output columns, which the products allow) so that the
//     mma.sync operand and accumulator fragments ARE the row-chunk layout -
//     no shuffles or shared-memory round trips between C, D and P;
//   * the Hadamard products for D (Algorithm 4) and the update are purely
//     per-lane; the prediction and the residual take two xor-shuffles.
// Zero padding of J_n, R up to K follows Sec. 4.2.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define FT_MAXN 10
#define FT_TILE 16

// Cache path of the factor-phase row gathers (rows that other warps write
// during the pass): 0 = L2 only (ld.global.cg), 1 = L1 and L2 (ld.global.ca),
// 2 = read-only path (ld.global.nc, as the paper's __ldg).  L1 caching keeps
// the Zipf-hot rows on the SM (L2-only gathers of hot rows were 4x slower on
// the Netflix-shaped workload); a row another SM wrote meanwhile may be read
// stale, which the Hogwild pass tolerates as the paper's __ldg reads do.
#ifndef FT_FACTOR_LOAD
#define FT_FACTOR_LOAD 1
#endif

namespace ft {

// MATH_TF32X3: FP32-accurate products on the TF32 tensor cores, each operand
// split into a TF32 head and a TF32 tail (x = hi + lo) and the product taken
// as lo.hi + hi.lo + hi.hi (the lo.lo term, ~2^-22 relative, is dropped);
// used by the prediction and error passes.
enum Math { MATH_FP32 = 0, MATH_TF32 = 1, MATH_BF16 = 2, MATH_TF32X3 = 3 };

// Latched device error bits (workspace word 0).
enum : int { ERRBIT_NONFINITE = 1, ERRBIT_INDEX = 2, ERRBIT_VALUE = 4, ERRBIT_TIMEOUT = 8 };

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- arguments
struct EpochArgs {
  const int32_t *idx[FT_MAXN];      // coordinates of the processed nonzeros
  float *A[FT_MAXN];                // factor matrices, row-major I_n x J_n
  const float *B[FT_MAXN];          // core matrices, row-major J_n x R
  const float *scale[FT_MAXN];      // per-row step multipliers or null
  int64_t I[FT_MAXN];               // mode sizes (coordinates are bounds-checked)
  int J[FT_MAXN];
  int offJ[FT_MAXN];                // prefix sums of J_n (delta row layout)
  int R;
  int sumJ;
  unsigned vecmask;                 // bit n: rows of mode n can be read as full 16-byte chunks
  unsigned vec4mask;                // bit n: J_n % 4 == 0 and a 16-byte aligned base, so every
                                    // 4-column group of a row is one 16-byte access
  const float *vals;                // values
  int64_t begin, end;               // processed nonzero range [begin, end)
  float lr, lam;
  float *delta;                     // deterministic mode: -grad rows, row m - begin
  float *partial;                   // core phase: per-CTA (sum, comp) of G
  float *pred;                      // predict: outputs (index m - begin)
  double *err_partial;              // errors: per-CTA (sum e^2, sum |e|)
  int *err;                         // latched error word
  // Hot-row cache of the Hogwild factor pass (see k_factor): idx[n][m] < 0
  // addresses cache slot -idx - 1; slots [hot_base[n], hot_base[n + 1]) hold
  // rows of mode n, and hot_rows[slot] is the slot's row.
  const int32_t *hot_rows;
  int hot_base[FT_MAXN + 1];
  int hot_cap;                      // slots in shared memory (0 = no cache)
  int hot_window;                   // write-back/refresh every hot_window x 128 nonzeros of a CTA
  // Per-CTA copy of the cached rows as the CTA last read them from global
  // memory ([grid][hot_cap][K] floats, workspace): the write-back adds the
  // CTA's own change (cache - copy), times the slot's weight, instead of
  // storing the row.
  float *hot_snap;
  const float *hot_weight;          // per slot (see build_hot_cache)
  // Storage scheme of the core pass: C^(n) = A^(n) B^(n) precomputed for
  // every row, row-major I_n x K (columns >= R are zero), or null.
  const float *cst[FT_MAXN];
  // BF16 copies of A^(n) read by the BF16 core pass (k_core_coop with
  // ROWS16): rows of K values, zeros past J_n, two values per word.
  const uint32_t *abf[FT_MAXN];
};

// Mode of a cache slot.
__device__ __forceinline__ int slot_mode(const EpochArgs &p, int slot, int N) {
  int n = 0;
  while (n + 1 < N && slot >= p.hot_base[n + 1]) ++n;
  return n;
}

// ------------------------------------------------------------- small helpers
__device__ __forceinline__ uint32_t to_tf32(float f) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
  return r;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Output-column permutation of an n-tile: logical column 8u + c of the
// accumulator is physical column pi(8u + c) = CPL*(c/2) + 2u + (c%2), so that
// accumulator elements (c = 2t, 2t+1) land in the lane's own chunk.
template <int K>
__device__ __forceinline__ int out_col(int u, int c) {
  return (K / 4) * (c >> 1) + 2 * u + (c & 1);
}

// M(k, col) of the two products a.B (which = 0: M = B, k = j, col = r) and
// d.B^T (which = 1: M = B^T, k = r, col = j), zero outside J_n x R.
__device__ __forceinline__ float core_entry(const float *__restrict__ Bn, int J, int R, int which,
                                            int k, int col) {
  if (which == 0) return (k < J && col < R) ? Bn[k * R + col] : 0.f;
  return (col < J && k < R) ? Bn[col * R + k] : 0.f;
}

// ----------------------------------------------- y = x . M on a warp tile
// x, y: [16 x K] in the row-chunk layout.  One table per (mode, product) in
// shared memory, filled once per CTA.
template <int K, int MATH>
struct Prod;

// Plain FP32 on the CUDA cores: the lane gathers the full rows of x by
// shuffles within its group of four and multiplies by its column chunk of M.
template <int K>
struct Prod<K, MATH_FP32> {
  static constexpr int CPL = K / 4;
  static constexpr int WORDS = K * K;  // floats per table
  __device__ static void fill(float *tab, const float *__restrict__ Bn, int J, int R, int which) {
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) tab[e] = core_entry(Bn, J, R, which, e / K, e % K);
  }
  __device__ static void run(const float (&x)[2][CPL], const float *tab, float (&y)[2][CPL], int lane) {
    const int t = lane & 3;
    const int base = lane & ~3;
#pragma unroll
    for (int q = 0; q < CPL; ++q) y[0][q] = y[1][q] = 0.f;
#pragma unroll
    for (int tt = 0; tt < 4; ++tt) {
#pragma unroll
      for (int qq = 0; qq < CPL; ++qq) {
        const float v0 = __shfl_sync(FULL, x[0][qq], base | tt);
        const float v1 = __shfl_sync(FULL, x[1][qq], base | tt);
        const float *row = tab + (CPL * tt + qq) * K + CPL * t;
        float m[CPL];
        if constexpr (CPL % 4 == 0) {
#pragma unroll
          for (int w = 0; w < CPL; w += 4) {
            const float4 f = *reinterpret_cast<const float4 *>(row + w);
            m[w] = f.x; m[w + 1] = f.y; m[w + 2] = f.z; m[w + 3] = f.w;
          }
        } else {
#pragma unroll
          for (int w = 0; w < CPL; ++w) m[w] = row[w];
        }
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
          y[0][q] = fmaf(v0, m[q], y[0][q]);
          y[1][q] = fmaf(v1, m[q], y[1][q]);
        }
      }
    }
  }
};

// TF32 tensor cores, mma.sync m16n8k8.  k-step s, lane (g, t): logical k = t
// is physical column CPL*t + 2s, logical k = t + 4 is CPL*t + 2s + 1.
template <int K>
struct Prod<K, MATH_TF32> {
  static constexpr int CPL = K / 4;
  static constexpr int NT = K / 8;   // n-tiles
  static constexpr int KS = K / 8;   // k-steps
  static constexpr int WORDS = NT * KS * 32 * 2;
  __device__ static void fill(float *tabf, const float *__restrict__ Bn, int J, int R, int which) {
    uint32_t *tab = reinterpret_cast<uint32_t *>(tabf);
    for (int e = threadIdx.x; e < NT * KS * 32; e += blockDim.x) {
      const int lane = e & 31, us = e >> 5, s = us % KS, u = us / KS;
      const int g = lane >> 2, t = lane & 3;
      const int col = out_col<K>(u, g);
      const int k0 = CPL * t + 2 * s;
      tab[2 * e] = to_tf32(core_entry(Bn, J, R, which, k0, col));
      tab[2 * e + 1] = to_tf32(core_entry(Bn, J, R, which, k0 + 1, col));
    }
  }
  __device__ static void run(const float (&x)[2][CPL], const float *tabf, float (&y)[2][CPL], int lane) {
    const uint2 *tab = reinterpret_cast<const uint2 *>(tabf);
    uint32_t xa[2][CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) { xa[0][q] = to_tf32(x[0][q]); xa[1][q] = to_tf32(x[1][q]); }
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int s = 0; s < KS; ++s) {
        const uint2 b = tab[(u * KS + s) * 32 + lane];
        mma_tf32(acc, xa[0][2 * s], xa[1][2 * s], xa[0][2 * s + 1], xa[1][2 * s + 1], b.x, b.y);
      }
      y[0][2 * u] = acc[0]; y[0][2 * u + 1] = acc[1];
      y[1][2 * u] = acc[2]; y[1][2 * u + 1] = acc[3];
    }
  }
};

// Three-pass TF32 (MATH_TF32X3) with the layout of Prod<K, MATH_TF32>: the
// table holds the head and the tail of every B fragment.
template <int K>
struct Prod<K, MATH_TF32X3> {
  static constexpr int CPL = K / 4;
  static constexpr int NT = K / 8;
  static constexpr int KS = K / 8;
  static constexpr int WORDS = NT * KS * 32 * 4;
  // x = hi + lo, each rounded to the 10 stored mantissa bits of TF32 to
  // nearest, ties away from zero (the rounding of cvt.rna.tf32.f32): adding
  // half a TF32 ulp (bit 12) to the bit pattern carries into the kept bits
  // exactly when the 13 dropped bits are at least half an ulp, and clearing
  // them truncates.  Two integer operations instead of the conversion's
  // longer sequence (the split is on the inner loops of every FP32-accurate
  // product).  For finite x below the float32 maximum the bits equal those of
  // cvt.rna; v - hi is exact in float32.
  __device__ static uint32_t round_bits(float v) { return (__float_as_uint(v) + 0x1000u) & 0xffffe000u; }
  __device__ static void split(float v, uint32_t &hi, uint32_t &lo) {
    hi = round_bits(v);
    lo = round_bits(v - __uint_as_float(hi));
  }
  __device__ static void fill(float *tabf, const float *__restrict__ Bn, int J, int R, int which) {
    uint32_t *tab = reinterpret_cast<uint32_t *>(tabf);
    for (int e = threadIdx.x; e < NT * KS * 32; e += blockDim.x) {
      const int lane = e & 31, us = e >> 5, s = us % KS, u = us / KS;
      const int g = lane >> 2, t = lane & 3;
      const int col = out_col<K>(u, g);
      const int k0 = CPL * t + 2 * s;
      split(core_entry(Bn, J, R, which, k0, col), tab[4 * e], tab[4 * e + 2]);
      split(core_entry(Bn, J, R, which, k0 + 1, col), tab[4 * e + 1], tab[4 * e + 3]);
    }
  }
  __device__ static void run(const float (&x)[2][CPL], const float *tabf, float (&y)[2][CPL], int lane) {
    const uint4 *tab = reinterpret_cast<const uint4 *>(tabf);
    if constexpr (K == 32) {
      // k-steps outside, n-tiles inside: only one k-step's split operands
      // are live (8 registers instead of 4 K), for the register-bound K = 32
      // tiles; per n-tile the three products of a k-step are added tail
      // terms first
      float acc[NT][4];
#pragma unroll
      for (int u = 0; u < NT; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.f;
#pragma unroll
      for (int s = 0; s < KS; ++s) {
        uint32_t h[4], l[4];
        split(x[0][2 * s], h[0], l[0]);
        split(x[1][2 * s], h[1], l[1]);
        split(x[0][2 * s + 1], h[2], l[2]);
        split(x[1][2 * s + 1], h[3], l[3]);
#pragma unroll
        for (int u = 0; u < NT; ++u) {
          const uint4 b = tab[(u * KS + s) * 32 + lane];
          mma_tf32(acc[u], l[0], l[1], l[2], l[3], b.x, b.y);
          mma_tf32(acc[u], h[0], h[1], h[2], h[3], b.z, b.w);
          mma_tf32(acc[u], h[0], h[1], h[2], h[3], b.x, b.y);
        }
      }
#pragma unroll
      for (int u = 0; u < NT; ++u) {
        y[0][2 * u] = acc[u][0]; y[0][2 * u + 1] = acc[u][1];
        y[1][2 * u] = acc[u][2]; y[1][2 * u + 1] = acc[u][3];
      }
      return;
    }
    uint32_t xh[2][CPL], xl[2][CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      split(x[0][q], xh[0][q], xl[0][q]);
      split(x[1][q], xh[1][q], xl[1][q]);
    }
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int s = 0; s < KS; ++s) {
        const uint4 b = tab[(u * KS + s) * 32 + lane];
        mma_tf32(acc, xl[0][2 * s], xl[1][2 * s], xl[0][2 * s + 1], xl[1][2 * s + 1], b.x, b.y);
        mma_tf32(acc, xh[0][2 * s], xh[1][2 * s], xh[0][2 * s + 1], xh[1][2 * s + 1], b.z, b.w);
      }
#pragma unroll
      for (int s = 0; s < KS; ++s) {
        const uint4 b = tab[(u * KS + s) * 32 + lane];
        mma_tf32(acc, xh[0][2 * s], xh[1][2 * s], xh[0][2 * s + 1], xh[1][2 * s + 1], b.x, b.y);
      }
      y[0][2 * u] = acc[0]; y[0][2 * u + 1] = acc[1];
      y[1][2 * u] = acc[2]; y[1][2 * u + 1] = acc[3];
    }
  }
};

// BF16 tensor cores, mma.sync m16n8k16.  k-step s, lane (g, t): logical
// k = 2t, 2t+1 are physical CPL*t + 4s + {0, 1}; k = 2t+8, 2t+9 are
// CPL*t + 4s + {2, 3}.
template <int K>
struct Prod<K, MATH_BF16> {
  static constexpr int CPL = K / 4;
  static constexpr int NT = K / 8;
  static constexpr int KS = K / 16;
  static constexpr int WORDS = NT * KS * 32 * 2;
  __device__ static void fill(float *tabf, const float *__restrict__ Bn, int J, int R, int which) {
    uint32_t *tab = reinterpret_cast<uint32_t *>(tabf);
    for (int e = threadIdx.x; e < NT * KS * 32; e += blockDim.x) {
      const int lane = e & 31, us = e >> 5, s = us % KS, u = us / KS;
      const int g = lane >> 2, t = lane & 3;
      const int col = out_col<K>(u, g);
      const int k0 = CPL * t + 4 * s;
      tab[2 * e] = pack_bf16(core_entry(Bn, J, R, which, k0, col), core_entry(Bn, J, R, which, k0 + 1, col));
      tab[2 * e + 1] =
          pack_bf16(core_entry(Bn, J, R, which, k0 + 2, col), core_entry(Bn, J, R, which, k0 + 3, col));
    }
  }
  __device__ static void run(const float (&x)[2][CPL], const float *tabf, float (&y)[2][CPL], int lane) {
    uint32_t xa[2][CPL / 2];
#pragma unroll
    for (int q = 0; q < CPL / 2; ++q) {
      xa[0][q] = pack_bf16(x[0][2 * q], x[0][2 * q + 1]);
      xa[1][q] = pack_bf16(x[1][2 * q], x[1][2 * q + 1]);
    }
    run_packed(xa, tabf, y, lane);
  }
  // x already rounded: word q of row h holds its columns CPL*t + 2q, + 1
  __device__ static void run_packed(const uint32_t (&xa)[2][CPL / 2], const float *tabf, float (&y)[2][CPL],
                                    int lane) {
    const uint2 *tab = reinterpret_cast<const uint2 *>(tabf);
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int s = 0; s < KS; ++s) {
        const uint2 b = tab[(u * KS + s) * 32 + lane];
        mma_bf16(acc, xa[0][2 * s], xa[1][2 * s], xa[0][2 * s + 1], xa[1][2 * s + 1], b.x, b.y);
      }
      y[0][2 * u] = acc[0]; y[0][2 * u + 1] = acc[1];
      y[1][2 * u] = acc[2]; y[1][2 * u + 1] = acc[3];
    }
  }
};

// ---------------------------------------------------------- row-chunk I/O
// Read the lane's chunk of factor row `row` (zeros past J_n or when !valid).
// In the factor phase rows are read at L2 (ld.global.cg) because other warps
// write them during the pass; the core phase may use the read-only path.
template <int K, bool READ_ONLY>
__device__ __forceinline__ void load_chunk(const float *__restrict__ An, int64_t row, int J, int t,
                                           bool valid, bool vec, bool vec4, float (&v)[K / 4]) {
  constexpr int CPL = K / 4;
  if (!valid) {
#pragma unroll
    for (int q = 0; q < CPL; ++q) v[q] = 0.f;
    return;
  }
  const float *p = An + row * J + CPL * t;
  if (vec) {
#pragma unroll
    for (int w = 0; w < CPL; w += 4) {
      float4 f;
      if constexpr (READ_ONLY || FT_FACTOR_LOAD == 2) f = __ldg(reinterpret_cast<const float4 *>(p + w));
      else if constexpr (FT_FACTOR_LOAD == 1) f = __ldca(reinterpret_cast<const float4 *>(p + w));
      else f = __ldcg(reinterpret_cast<const float4 *>(p + w));
      v[w] = f.x; v[w + 1] = f.y; v[w + 2] = f.z; v[w + 3] = f.w;
    }
  } else if (vec4) {
    // rows narrower than K: the 4-column groups inside the row, one 16-byte
    // load each (J_n is a multiple of 4, so a group is wholly in or out)
#pragma unroll
    for (int w = 0; w < CPL; w += 4) {
      float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
      if (CPL * t + w < J) {
        if constexpr (READ_ONLY || FT_FACTOR_LOAD == 2) f = __ldg(reinterpret_cast<const float4 *>(p + w));
        else if constexpr (FT_FACTOR_LOAD == 1) f = __ldca(reinterpret_cast<const float4 *>(p + w));
        else f = __ldcg(reinterpret_cast<const float4 *>(p + w));
      }
      v[w] = f.x; v[w + 1] = f.y; v[w + 2] = f.z; v[w + 3] = f.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      const int j = CPL * t + q;
      if (j < J) v[q] = (READ_ONLY || FT_FACTOR_LOAD == 2) ? __ldg(p + q)
                        : (FT_FACTOR_LOAD == 1 ? __ldca(p + q) : __ldcg(p + q));
      else v[q] = 0.f;
    }
  }
}

template <int K>
__device__ __forceinline__ void store_chunk(float *__restrict__ An, int64_t row, int J, int t, bool vec,
                                            bool vec4, const float (&v)[K / 4]) {
  constexpr int CPL = K / 4;
  float *p = An + row * J + CPL * t;
  if (vec) {
#pragma unroll
    for (int w = 0; w < CPL; w += 4) __stcg(reinterpret_cast<float4 *>(p + w), make_float4(v[w], v[w + 1], v[w + 2], v[w + 3]));
  } else if (vec4) {
#pragma unroll
    for (int w = 0; w < CPL; w += 4)
      if (CPL * t + w < J) __stcg(reinterpret_cast<float4 *>(p + w), make_float4(v[w], v[w + 1], v[w + 2], v[w + 3]));
  } else {
#pragma unroll
    for (int q = 0; q < CPL; ++q)
      if (CPL * t + q < J) __stcg(p + q, v[q]);
  }
}

// The lane's chunk of row `row` of a BF16 row copy (rows of K values, two per
// word): K/8 words, zeros when !valid.
template <int K>
__device__ __forceinline__ void load_chunk_bf16(const uint32_t *__restrict__ Abf, int64_t row, int t,
                                                bool valid, uint32_t (&v)[K / 8]) {
  const uint32_t *src = Abf + row * (K / 2) + (K / 8) * t;
  if constexpr (K == 16) {
    uint2 w = make_uint2(0u, 0u);
    if (valid) w = __ldg(reinterpret_cast<const uint2 *>(src));
    v[0] = w.x; v[1] = w.y;
  } else {
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    if (valid) w = __ldg(reinterpret_cast<const uint4 *>(src));
    v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
  }
}

// Coordinates and values of one warp tile (loaded a tile ahead of use).
template <int N>
struct TileCoords {
  int64_t m[2];
  bool valid[2];
  int32_t row[N][2];
  float x[2];

  __device__ __forceinline__ void load(const EpochArgs &p, int64_t tile_base, int lane, bool need_x) {
    const int g = lane >> 2;
    m[0] = tile_base + g;
    m[1] = tile_base + g + 8;
    valid[0] = m[0] < p.end;
    valid[1] = m[1] < p.end;
#pragma unroll
    for (int n = 0; n < N; ++n)
#pragma unroll
      for (int h = 0; h < 2; ++h) row[n][h] = valid[h] ? __ldcs(p.idx[n] + m[h]) : 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) x[h] = (need_x && valid[h]) ? __ldcs(p.vals + m[h]) : 0.f;
  }
};

// ------------------------------------------------------- shared tile front
// Gathers the tile (a1, a2), forms C^(n) = A_Psi^(n) B^(n) for every mode
// (Algorithm 4, C step) and the prediction xhat per row (Eq. "fasttucker").
template <int N, int K, int MATH, bool READ_ONLY>
struct Front {
  static constexpr int CPL = K / 4;
  int64_t m[2];
  bool valid[2];
  int32_t row[N][2];                // global row, or cache slot when hot
  unsigned hot;                     // bit 2n + h: row[n][h] is a cache slot
  float x[2];
  float a[N][2][CPL];
  float c[N][2][CPL];
  float xhat[2];

  // rep: the CTA's hot-row cache ([hot_cap][K] floats) or null.
  __device__ __forceinline__ void load(const EpochArgs &p, int64_t tile_base, int lane, bool need_x,
                                       const float *rep = nullptr) {
    TileCoords<N> tc;
    tc.load(p, tile_base, lane, need_x);
    gather(p, tc, lane, rep);
  }

  // Decode the coordinates (bounds, cache slots) and gather the rows.
  // rows = false: decode only (the caller reads the rows from elsewhere).
  __device__ __forceinline__ void gather(const EpochArgs &p, const TileCoords<N> &tc, int lane,
                                         const float *rep = nullptr, bool rows = true) {
    const int t = lane & 3;
    hot = 0u;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      m[h] = tc.m[h];
      valid[h] = tc.valid[h];
      x[h] = tc.x[h];
    }
#pragma unroll
    for (int n = 0; n < N; ++n)
#pragma unroll
      for (int h = 0; h < 2; ++h) row[n][h] = tc.row[n][h];
    // a coordinate outside [0, I_n) (or a slot outside the cache) masks its
    // nonzero and latches an error
    bool bad = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      bool ok = true;
#pragma unroll
      for (int n = 0; n < N; ++n) {
        const int32_t v = row[n][h];
        if (rep != nullptr && v < 0) {
          ok = ok && (-v - 1) >= p.hot_base[n] && (-v - 1) < p.hot_base[n + 1];
          row[n][h] = -v - 1;
          hot |= 1u << (2 * n + h);
        } else {
          ok = ok && v >= 0 && int64_t(v) < p.I[n];
        }
      }
      if (valid[h] && !ok) {
        bad = true;
        valid[h] = false;
#pragma unroll
        for (int n = 0; n < N; ++n) row[n][h] = 0;
        hot &= ~((0x55555555u) << h);
      }
    }
    if (bad) atomicOr(p.err, ERRBIT_INDEX);
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (!valid[h]) x[h] = 0.f;
    if (!rows) return;
#pragma unroll
    for (int n = 0; n < N; ++n)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const bool is_hot = (hot >> (2 * n + h)) & 1u;
        if (rep != nullptr && ((p.vecmask >> n) & 1) != 0) {
          // full-width rows: one generic 16-byte load from the cache or from
          // global memory (a select, not a divergent branch)
          const float *src = is_hot ? rep + size_t(row[n][h]) * K + CPL * t
                                    : p.A[n] + int64_t(row[n][h]) * p.J[n] + CPL * t;
#pragma unroll
          for (int w = 0; w < CPL; w += 4) {
            float4 f4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (valid[h]) f4 = *reinterpret_cast<const float4 *>(src + w);
            a[n][h][w] = f4.x; a[n][h][w + 1] = f4.y; a[n][h][w + 2] = f4.z; a[n][h][w + 3] = f4.w;
          }
        } else if (is_hot) {
          const float *src = rep + size_t(row[n][h]) * K + CPL * t;
#pragma unroll
          for (int w = 0; w < CPL; w += 4) {
            const float4 f4 = *reinterpret_cast<const float4 *>(src + w);
            a[n][h][w] = f4.x; a[n][h][w + 1] = f4.y; a[n][h][w + 2] = f4.z; a[n][h][w + 3] = f4.w;
          }
        } else {
          load_chunk<K, READ_ONLY>(p.A[n], row[n][h], p.J[n], t, valid[h], (p.vecmask >> n) & 1,
                                   (p.vec4mask >> n) & 1, a[n][h]);
        }
      }
  }

  __device__ __forceinline__ void compute(const float *tabB, int tab_words, int lane) {
    // tabB: table of product a.B of mode n at tabB + n * tab_words
#pragma unroll
    for (int n = 0; n < N; ++n) Prod<K, MATH>::run(a[n], tabB + n * tab_words, c[n], lane);
    predict();
  }

  // Storage scheme (Sec. 5.6, "Replace memory access with calculation"): the
  // rows of C^(n) = A^(n) B^(n) are read from p.cst instead of formed here.
  __device__ __forceinline__ void load_stored(const EpochArgs &p, int lane) {
    const int t = lane & 3;
#pragma unroll
    for (int n = 0; n < N; ++n)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float *src = p.cst[n] + int64_t(row[n][h]) * K + CPL * t;
#pragma unroll
        for (int w = 0; w < CPL; w += 4) {
          float4 f4 = make_float4(0.f, 0.f, 0.f, 0.f);
          if (valid[h]) f4 = __ldg(reinterpret_cast<const float4 *>(src + w));
          c[n][h][w] = f4.x; c[n][h][w + 1] = f4.y; c[n][h][w + 2] = f4.z; c[n][h][w + 3] = f4.w;
        }
      }
    predict();
  }

  __device__ __forceinline__ void predict() {
    // xhat = sum_r prod_n c^(n)_r: lane partial over its chunk (the last
    // factor of each product fused into the sum), then the group of four
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        if constexpr (N == 1) {
          s += c[0][h][q];
        } else {
          float pr = c[0][h][q];
#pragma unroll
          for (int n = 1; n + 1 < N; ++n) pr *= c[n][h][q];
          s = fmaf(pr, c[N - 1][h][q], s);
        }
      }
      s += __shfl_xor_sync(FULL, s, 1);
      s += __shfl_xor_sync(FULL, s, 2);
      xhat[h] = s;
    }
  }

  // D^(n) = prod_{k != n} C^(k) (Algorithm 4, Hadamard step)
  __device__ __forceinline__ void leave_one_out(int n, float (&d)[2][CPL]) const {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        float pr = 1.f;
#pragma unroll
        for (int k = 0; k < N; ++k)
          if (k != n) pr *= c[k][h][q];
        d[h][q] = pr;
      }
  }
};

// Shared-memory layout of the factor kernel: for each mode the a.B table,
// then for each mode the d.B^T table, then (Hogwild pass) the hot-row cache
// [hot_cap][K] floats and its dirty flags [hot_cap] bytes.
template <int N, int K, int MATH>
struct FactorSmem {
  static constexpr int TW = Prod<K, MATH>::WORDS;
  static constexpr size_t tables() { return size_t(2) * N * TW * sizeof(float); }
};

template <int N, int K, int MATH>
__device__ __forceinline__ void fill_tables(float *smem, const EpochArgs &p, bool both) {
  constexpr int TW = Prod<K, MATH>::WORDS;
#pragma unroll 1
  for (int n = 0; n < N; ++n) {
    Prod<K, MATH>::fill(smem + n * TW, p.B[n], p.J[n], p.R, 0);
    if (both) Prod<K, MATH>::fill(smem + (N + n) * TW, p.B[n], p.J[n], p.R, 1);
  }
}

// Hot-row cache traffic (whole CTA).  Refresh: copy every slot from L2 into
// the cache and into the CTA's snapshot (global, private to the CTA).
// Write-back: for every dirty slot add w_slot (cache - snapshot) - the CTA's
// own change of the row since the refresh, weighted - to the global row with
// float atomics, then clear the flags.  No CTA overwrites another CTA's
// change.  w_slot = 1 (Hogwild: the CTAs' steps add up) for rows a CTA meets
// less than once per window; for rows every CTA meets many times per window
// w_slot = 1 / (CTAs expected to change the row in one window), so the row
// moves by the average of the CTAs' changes (parameter averaging): each CTA
// has run the row toward the same optimum on its own share of the data, and
// their sum would overshoot it by that many times.
template <int K>
__device__ __forceinline__ float *cta_snapshot(const EpochArgs &p) {
  return p.hot_snap + size_t(blockIdx.x) * size_t(p.hot_cap) * K;
}

template <int N, int K>
__device__ void cache_refresh(const EpochArgs &p, float *rep) {
  float *snap = cta_snapshot<K>(p);
  for (int e = threadIdx.x; e < p.hot_cap * (K / 4); e += blockDim.x) {
    const int slot = e / (K / 4), j0 = 4 * (e % (K / 4));
    const int n = slot_mode(p, slot, N);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (slot < p.hot_base[N] && j0 < p.J[n]) {
      const float *src = p.A[n] + int64_t(__ldg(p.hot_rows + slot)) * p.J[n] + j0;
      if (((p.vec4mask >> n) & 1) != 0) {
        v = __ldcg(reinterpret_cast<const float4 *>(src));
      } else {
        v.x = __ldcg(src);
        if (j0 + 1 < p.J[n]) v.y = __ldcg(src + 1);
        if (j0 + 2 < p.J[n]) v.z = __ldcg(src + 2);
        if (j0 + 3 < p.J[n]) v.w = __ldcg(src + 3);
      }
    }
    *reinterpret_cast<float4 *>(rep + size_t(slot) * K + j0) = v;
    __stcg(reinterpret_cast<float4 *>(snap + size_t(slot) * K + j0), v);
  }
}

template <int N, int K>
__device__ void cache_write_back(const EpochArgs &p, const float *rep, unsigned char *dirty) {
  const float *snap = cta_snapshot<K>(p);
  for (int e = threadIdx.x; e < p.hot_cap * (K / 4); e += blockDim.x) {
    const int slot = e / (K / 4), j0 = 4 * (e % (K / 4));
    const int n = slot_mode(p, slot, N);
    if (slot >= p.hot_base[N] || j0 >= p.J[n] || !dirty[slot]) continue;
    const float4 v = *reinterpret_cast<const float4 *>(rep + size_t(slot) * K + j0);
    const float4 s = __ldcg(reinterpret_cast<const float4 *>(snap + size_t(slot) * K + j0));
    const float w = __ldg(p.hot_weight + slot);
    const float4 d = make_float4(w * (v.x - s.x), w * (v.y - s.y), w * (v.z - s.z), w * (v.w - s.w));
    float *dst = p.A[n] + int64_t(__ldg(p.hot_rows + slot)) * p.J[n] + j0;
    if (((p.vec4mask >> n) & 1) != 0) {
      atomicAdd(reinterpret_cast<float4 *>(dst), d);
    } else {
      atomicAdd(dst, d.x);
      if (j0 + 1 < p.J[n]) atomicAdd(dst + 1, d.y);
      if (j0 + 2 < p.J[n]) atomicAdd(dst + 2, d.z);
      if (j0 + 3 < p.J[n]) atomicAdd(dst + 3, d.w);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < p.hot_cap; e += blockDim.x) dirty[e] = 0;
}

// One factor-phase tile (Algorithm 4): C = A_Psi B, D = *_{k != n} C,
// P = D B^T, e = x - xhat, then per mode either the new rows
//   a <- a + lr * s_row * (e P - lam a)   (Eq. "Update_FastTuckerPlus_factor")
// are stored (Hogwild; hot rows go to the CTA's cache), or (DELTA) the
// per-nonzero step e P - lam a is written for the deterministic reduction.
template <int N, int K, int MATH, bool DELTA>
__device__ __forceinline__ void factor_tile(const EpochArgs &p, const float *tabs, float *rep,
                                            unsigned char *dirty, const TileCoords<N> &tc, int lane) {
  constexpr int CPL = K / 4;
  constexpr int TW = Prod<K, MATH>::WORDS;
  const int t = lane & 3;
  Front<N, K, MATH, false> f;
  f.gather(p, tc, lane, rep);
  f.compute(tabs, TW, lane);
  float e[2];
  e[0] = f.x[0] - f.xhat[0];
  e[1] = f.x[1] - f.xhat[1];
  const bool bad = (f.valid[0] && !isfinite(e[0])) || (f.valid[1] && !isfinite(e[1]));
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(p.err, ERRBIT_NONFINITE);
#pragma unroll
  for (int n = 0; n < N; ++n) {
    float d[2][CPL], pp[2][CPL];
    f.leave_one_out(n, d);
    Prod<K, MATH>::run(d, tabs + (N + n) * TW, pp, lane);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!f.valid[h]) continue;
      float out[CPL];
      if constexpr (DELTA) {
#pragma unroll
        for (int q = 0; q < CPL; ++q) out[q] = e[h] * pp[h][q] - p.lam * f.a[n][h][q];
        float *dst = p.delta + (f.m[h] - p.begin) * p.sumJ + p.offJ[n] + CPL * t;
#pragma unroll
        for (int q = 0; q < CPL; ++q)
          if (CPL * t + q < p.J[n]) dst[q] = out[q];
      } else {
        const bool is_hot = (f.hot >> (2 * n + h)) & 1u;
        float lr = p.lr;
        if (p.scale[n]) {
          const int64_t grow = is_hot ? int64_t(__ldg(p.hot_rows + f.row[n][h])) : int64_t(f.row[n][h]);
          lr *= __ldg(p.scale[n] + grow);
        }
#pragma unroll
        for (int q = 0; q < CPL; ++q)
          out[q] = fmaf(lr, fmaf(e[h], pp[h][q], -p.lam * f.a[n][h][q]), f.a[n][h][q]);
        if (rep != nullptr && ((p.vecmask >> n) & 1) != 0) {
          // one generic 16-byte store to the cache or to global memory
          float *dst = is_hot ? rep + size_t(f.row[n][h]) * K + CPL * t
                              : p.A[n] + int64_t(f.row[n][h]) * p.J[n] + CPL * t;
#pragma unroll
          for (int w = 0; w < CPL; w += 4)
            *reinterpret_cast<float4 *>(dst + w) = make_float4(out[w], out[w + 1], out[w + 2], out[w + 3]);
          if (is_hot && t == 0) dirty[f.row[n][h]] = 1;
        } else if (is_hot) {
          float *dst = rep + size_t(f.row[n][h]) * K + CPL * t;
#pragma unroll
          for (int w = 0; w < CPL; w += 4)
            *reinterpret_cast<float4 *>(dst + w) = make_float4(out[w], out[w + 1], out[w + 2], out[w + 3]);
          if (t == 0) dirty[f.row[n][h]] = 1;
        } else {
          store_chunk<K>(p.A[n], f.row[n][h], p.J[n], t, (p.vecmask >> n) & 1, (p.vec4mask >> n) & 1, out);
        }
      }
    }
  }
}

// The Hogwild tile of factor_tile for the common case - every mode's rows
// exactly K wide with a 16-byte aligned base (so every chunk is one 16-byte
// access), the hot-row cache on, one step size for every row - with the same
// rule and no data-dependent branches: a masked nonzero (past the end, or with
// a coordinate outside its range) reads row 0 of global memory, uses zeros,
// and skips its stores by predication.  The update is the step of
// a + lr (e P - lam a), written for FP32-accurate products as
//   a <- a + ((lr e) P + (-lr lam) a)
// (the step is formed first, so the row is rounded once, by the final add),
// and for TF32/BF16 products, whose rounding (2^-11, 2^-8 of the products)
// dwarfs a few float32 roundings of the row, as the two operations
//   a <- (1 - lr lam) a + (lr e) P.
// NARROW: rows J_n < K wide (J_n a multiple of 4, 16-byte aligned base): the
// global rows have stride J_n and only the 4-column groups inside the row are
// read and written; cached rows stay K wide (zeros past J_n, and the products
// leave them zero).  Without the cache (rep null) every coordinate is a
// global row.
template <int N, int K, int MATH, bool NARROW = false>
__device__ __forceinline__ void factor_tile_fast(const EpochArgs &p, const float *tabs, float *rep,
                                                 unsigned char *dirty, const TileCoords<N> &tc, int lane) {
  constexpr int CPL = K / 4;
  constexpr int TW = Prod<K, MATH>::WORDS;
  const int t = lane & 3;
  Front<N, K, MATH, false> f;
  uint32_t r[N][2];      // global row, or cache slot when hot
  bool hot[N][2];
  bool bad = false;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    bool ok = true;
#pragma unroll
    for (int n = 0; n < N; ++n) {
      const int32_t v = tc.row[n][h];
      const bool is_hot = v < 0;
      const uint32_t slot = ~uint32_t(v);   // -v - 1 for a negative v
      const bool in = is_hot ? slot - uint32_t(p.hot_base[n]) < uint32_t(p.hot_base[n + 1] - p.hot_base[n])
                             : uint32_t(v) < uint32_t(p.I[n]);
      ok = ok && in;
      hot[n][h] = is_hot;
      r[n][h] = is_hot ? slot : uint32_t(v);
    }
    bad = bad || (tc.valid[h] && !ok);
    f.valid[h] = tc.valid[h] && ok;
    f.x[h] = f.valid[h] ? tc.x[h] : 0.f;
#pragma unroll
    for (int n = 0; n < N; ++n) {
      hot[n][h] = hot[n][h] && f.valid[h];
      r[n][h] = f.valid[h] ? r[n][h] : 0u;
    }
  }
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(p.err, ERRBIT_INDEX);
  // gather: one generic 16-byte access per chunk, from the cache or from
  // global memory (masked rows read row 0 and use zeros)
#pragma unroll
  for (int n = 0; n < N; ++n)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const size_t stride = NARROW ? size_t(p.J[n]) : size_t(K);
      const float *src = hot[n][h] ? rep + r[n][h] * K + CPL * t : p.A[n] + size_t(r[n][h]) * stride + CPL * t;
#pragma unroll
      for (int w = 0; w < CPL; w += 4) {
        float4 f4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!NARROW || hot[n][h] || CPL * t + w < p.J[n]) f4 = *reinterpret_cast<const float4 *>(src + w);
        f.a[n][h][w] = f.valid[h] ? f4.x : 0.f;
        f.a[n][h][w + 1] = f.valid[h] ? f4.y : 0.f;
        f.a[n][h][w + 2] = f.valid[h] ? f4.z : 0.f;
        f.a[n][h][w + 3] = f.valid[h] ? f4.w : 0.f;
      }
    }
  f.compute(tabs, TW, lane);
  const float e[2] = {f.x[0] - f.xhat[0], f.x[1] - f.xhat[1]};
  const bool nonfinite = (f.valid[0] && !isfinite(e[0])) || (f.valid[1] && !isfinite(e[1]));
  if (__any_sync(FULL, nonfinite) && lane == 0) atomicOr(p.err, ERRBIT_NONFINITE);
  constexpr bool ROUND_ONCE = MATH == MATH_FP32 || MATH == MATH_TF32X3;
  const float nl = -p.lr * p.lam;
  const float keep = 1.f - p.lr * p.lam;
  const float ge[2] = {p.lr * e[0], p.lr * e[1]};
#pragma unroll
  for (int n = 0; n < N; ++n) {
    float d[2][CPL], pp[2][CPL];
    f.leave_one_out(n, d);
    Prod<K, MATH>::run(d, tabs + (N + n) * TW, pp, lane);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const size_t stride = NARROW ? size_t(p.J[n]) : size_t(K);
      float *dst = hot[n][h] ? rep + r[n][h] * K + CPL * t : p.A[n] + size_t(r[n][h]) * stride + CPL * t;
#pragma unroll
      for (int w = 0; w < CPL; w += 4) {
        float4 o;
        if constexpr (ROUND_ONCE)
          o = make_float4(f.a[n][h][w] + fmaf(ge[h], pp[h][w], nl * f.a[n][h][w]),
                          f.a[n][h][w + 1] + fmaf(ge[h], pp[h][w + 1], nl * f.a[n][h][w + 1]),
                          f.a[n][h][w + 2] + fmaf(ge[h], pp[h][w + 2], nl * f.a[n][h][w + 2]),
                          f.a[n][h][w + 3] + fmaf(ge[h], pp[h][w + 3], nl * f.a[n][h][w + 3]));
        else
          o = make_float4(fmaf(ge[h], pp[h][w], keep * f.a[n][h][w]),
                          fmaf(ge[h], pp[h][w + 1], keep * f.a[n][h][w + 1]),
                          fmaf(ge[h], pp[h][w + 2], keep * f.a[n][h][w + 2]),
                          fmaf(ge[h], pp[h][w + 3], keep * f.a[n][h][w + 3]));
        if (f.valid[h] && (!NARROW || hot[n][h] || CPL * t + w < p.J[n]))
          *reinterpret_cast<float4 *>(dst + w) = o;
      }
      if (hot[n][h] && t == 0) dirty[r[n][h]] = 1;
    }
  }
}

// ------------------------------------------------------------- factor phase
// One pass of the factor update over [begin, end) (Algorithm 4).
//
// DELTA = false (Hogwild, as the paper's kernel): rows are stored back as soon
// as a tile is done.  Rows that many nonzeros share are the costly ones on
// GB300 - every store to a line that other SMs keep reading turns their
// next reads into slow coherence misses, and the stores themselves queue on
// the hottest lines.  So the hottest rows of every mode (chosen at ft_init
// from the row counts) live in a per-CTA write-back cache in shared memory:
// the CTA's warps read and update the cached copy, and after every
// hot_window x 128 of its nonzeros the CTA adds its weighted change of every
// dirty row to global memory
// (float atomics, so no CTA overwrites another's change; see
// cache_write_back) and refreshes its copy.
// Rows outside the cache are stored back with plain stores: concurrent
// updates of one of them may be lost, as in the paper's kernel.
// Coordinates of cached rows arrive remapped to -(slot + 1); the slots are
// shared by all modes and go to the most frequent rows of the tensor.
//
// DELTA = true: the per-nonzero step is written to p.delta for the
// deterministic batch reduction; A is not modified.
// FAST (Hogwild with the hot-row cache, every mode full width, one step size
// for every row): the tiles run factor_tile_fast; FAST and NARROW: the same
// where every mode's rows are read as 16-byte groups but some are narrower
// than K.
//
// CTA shape: where the tile fits in 128 registers (K = 16, N <= 3) the
// cached Hogwild pass runs one 512-thread CTA per SM, so the SM's shared
// memory holds one cache of twice the rows instead of two CTAs' copies of
// the same rows; elsewhere two (or one) 256-thread CTAs per SM.  The window
// is counted in the CTA's nonzeros: a write-back every hot_window x 128 of
// them, rounded up to whole CTA tiles.
template <int N, int K, int MATH>
struct FactorLaunch {
  static constexpr int THREADS = (K == 16 && N <= 3) ? 512 : 256;
};

template <int N, int K, int MATH, bool DELTA, bool FAST = false, bool NARROW = false>
__global__ void __launch_bounds__(FactorLaunch<N, K, MATH>::THREADS) k_factor(const EpochArgs p) {
  extern __shared__ __align__(16) float smem[];
  using L = FactorSmem<N, K, MATH>;
  fill_tables<N, K, MATH>(smem, p, true);
  const bool cache = !DELTA && p.hot_cap > 0;
  float *rep = cache ? smem + 2 * N * L::TW : nullptr;
  unsigned char *dirty = cache ? reinterpret_cast<unsigned char *>(rep + size_t(p.hot_cap) * K) : nullptr;
  if (cache) {
    cache_refresh<N, K>(p, rep);
    for (int e = threadIdx.x; e < p.hot_cap; e += blockDim.x) dirty[e] = 0;
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int wpc = blockDim.x >> 5;
  const int64_t ntiles = (p.end - p.begin + FT_TILE - 1) / FT_TILE;
  // Each warp loads the coordinates and values of its next tile before it
  // works on the current one, so the stream's DRAM latency overlaps compute.
  if (!cache) {
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    TileCoords<N> cur, nxt;
    if (warp < ntiles) cur.load(p, p.begin + warp * FT_TILE, lane, true);
    for (int64_t tile = warp; tile < ntiles; tile += nwarps) {
      const int64_t next = tile + nwarps;
      if (next < ntiles) nxt.load(p, p.begin + next * FT_TILE, lane, true);
      factor_tile<N, K, MATH, DELTA>(p, smem, nullptr, nullptr, cur, lane);
      cur = nxt;
    }
    return;
  }
  // CTA tile c = warp tiles [c * wpc, c * wpc + wpc); CTA b takes c = b, b + G, ...
  const int64_t nct = (ntiles + wpc - 1) / wpc;
  const int64_t G = gridDim.x;
  const int W = p.hot_window > 0 ? (p.hot_window * 128 + wpc * FT_TILE - 1) / (wpc * FT_TILE) : 1;
  const int wid = threadIdx.x >> 5;
  TileCoords<N> cur, nxt;
  if (blockIdx.x < nct) cur.load(p, p.begin + (int64_t(blockIdx.x) * wpc + wid) * FT_TILE, lane, true);
  int k = 0;
  for (int64_t c = blockIdx.x; c < nct; c += G) {
    const int64_t cn = c + G;
    if (cn < nct) nxt.load(p, p.begin + (cn * wpc + wid) * FT_TILE, lane, true);
    if (c * wpc + wid < ntiles) {
      if constexpr (FAST) factor_tile_fast<N, K, MATH, NARROW>(p, smem, rep, dirty, cur, lane);
      else factor_tile<N, K, MATH, false>(p, smem, rep, dirty, cur, lane);
    }
    cur = nxt;
    if (++k == W || cn >= nct) {
      k = 0;
      __syncthreads();
      cache_write_back<N, K>(p, rep, dirty);
      if (cn < nct) {
        __syncthreads();
        cache_refresh<N, K>(p, rep);
        __syncthreads();
      }
    }
  }
}

// --------------------------------------------------------------- core phase
// Per tile: E^(n) = (xhat - x) * A_Psi^(n), G^(n) += E^(n)T D^(n) (Algorithm 5).
// The 16 x K operands are staged in the warp's shared memory so that the
// contraction over the tile's nonzeros can run on the tensor cores; the
// tile results are added with Neumaier compensation into per-warp float
// accumulators (lane-private slots), combined per CTA in warp order and
// written as one (sum, compensation) partial per CTA.  Fixed grid and static
// tile order make the result reproducible bit for bit.
//
// Accumulator slot q of a lane (q < K*K/32): q = (mt * (K/8) + u) * 4 + i is
// element (j, r) = (16 mt + g + 8 (i / 2), 8 u + 2 t + i % 2) of G^(n).
template <int K, int MATH>
struct GradTile {
  static constexpr int LD = (MATH == MATH_BF16) ? K + 4 : K + 8;  // conflict-free strides
  static constexpr int SLOTS = K * K / 32;
  __device__ static void run(const float *Es, const float *Ds, float (&out)[SLOTS], int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < K / 16; ++mt)
#pragma unroll
      for (int u = 0; u < K / 8; ++u) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const int j0 = 16 * mt + g, r0 = 8 * u + g;
        if constexpr (MATH == MATH_TF32) {
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            const int m0 = 8 * s + t, m1 = m0 + 4;
            mma_tf32(acc, to_tf32(Es[m0 * LD + j0]), to_tf32(Es[m0 * LD + j0 + 8]), to_tf32(Es[m1 * LD + j0]),
                     to_tf32(Es[m1 * LD + j0 + 8]), to_tf32(Ds[m0 * LD + r0]), to_tf32(Ds[m1 * LD + r0]));
          }
        } else if constexpr (MATH == MATH_BF16) {
          const int m0 = 2 * t, m2 = 2 * t + 8;
          mma_bf16(acc, pack_bf16(Es[m0 * LD + j0], Es[(m0 + 1) * LD + j0]),
                   pack_bf16(Es[m0 * LD + j0 + 8], Es[(m0 + 1) * LD + j0 + 8]),
                   pack_bf16(Es[m2 * LD + j0], Es[(m2 + 1) * LD + j0]),
                   pack_bf16(Es[m2 * LD + j0 + 8], Es[(m2 + 1) * LD + j0 + 8]),
                   pack_bf16(Ds[m0 * LD + r0], Ds[(m0 + 1) * LD + r0]),
                   pack_bf16(Ds[m2 * LD + r0], Ds[(m2 + 1) * LD + r0]));
        } else {
          // FP32: three-pass TF32 (x = hi + lo; lo.hi + hi.lo + hi.hi), the
          // same fragments as the TF32 path, FP32-accurate
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            const int m0 = 8 * s + t, m1 = m0 + 4;
            uint32_t ah[4], al[4], bh[2], bl[2];
            Prod<K, MATH_TF32X3>::split(Es[m0 * LD + j0], ah[0], al[0]);
            Prod<K, MATH_TF32X3>::split(Es[m0 * LD + j0 + 8], ah[1], al[1]);
            Prod<K, MATH_TF32X3>::split(Es[m1 * LD + j0], ah[2], al[2]);
            Prod<K, MATH_TF32X3>::split(Es[m1 * LD + j0 + 8], ah[3], al[3]);
            Prod<K, MATH_TF32X3>::split(Ds[m0 * LD + r0], bh[0], bl[0]);
            Prod<K, MATH_TF32X3>::split(Ds[m1 * LD + r0], bh[1], bl[1]);
            mma_tf32(acc, al[0], al[1], al[2], al[3], bh[0], bh[1]);
            mma_tf32(acc, ah[0], ah[1], ah[2], ah[3], bl[0], bl[1]);
            mma_tf32(acc, ah[0], ah[1], ah[2], ah[3], bh[0], bh[1]);
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) out[(mt * (K / 8) + u) * 4 + i] = acc[i];
      }
  }
};

__device__ __forceinline__ void neumaier_add(float &sum, float &comp, float v) {
  const float t = sum + v;
  if (fabsf(sum) >= fabsf(v)) comp += (sum - t) + v;
  else comp += (v - t) + sum;
  sum = t;
}

template <int N, int K, int MATH>
struct CoreSmem {
  static constexpr int TW = Prod<K, MATH>::WORDS;
  static constexpr int LD = GradTile<K, MATH>::LD;
  static constexpr int STAGE = 2 * FT_TILE * LD;          // floats per warp (E and D)
  static constexpr int ACC = 2 * N * K * K;               // floats per warp (sum and comp)
  static constexpr int WARPS = (N * K * K > 2048) ? 4 : 8;
  static constexpr size_t bytes() {
    return sizeof(float) * (size_t(N) * TW + size_t(WARPS) * (STAGE + ACC));
  }
};

// STORE: the storage scheme (rows of C read from p.cst, Sec. 5.6).
template <int N, int K, int MATH, bool STORE = false>
__global__ void __launch_bounds__(256) k_core(const EpochArgs p) {
  extern __shared__ __align__(16) float smem[];
  using L = CoreSmem<N, K, MATH>;
  constexpr int CPL = K / 4;
  constexpr int TW = L::TW;
  constexpr int LD = L::LD;
  constexpr int SL = GradTile<K, MATH>::SLOTS;
  fill_tables<N, K, MATH>(smem, p, false);
  const int warp_in_cta = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  float *stage = smem + N * TW + warp_in_cta * (L::STAGE + L::ACC);
  float *Es = stage, *Ds = stage + FT_TILE * LD;
  float *acc_s = stage + L::STAGE;            // [N][SL][32]
  float *acc_c = acc_s + N * SL * 32;
  for (int q = lane; q < N * SL * 32; q += 32) { acc_s[q] = 0.f; acc_c[q] = 0.f; }
  __syncthreads();

  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t ntiles = (p.end - p.begin + FT_TILE - 1) / FT_TILE;
  for (int64_t tile = warp; tile < ntiles; tile += nwarps) {
    Front<N, K, MATH, true> f;
    f.load(p, p.begin + tile * FT_TILE, lane, true);
    if constexpr (STORE) f.load_stored(p, lane);
    else f.compute(smem, TW, lane);
    const float ne0 = f.xhat[0] - f.x[0], ne1 = f.xhat[1] - f.x[1];
    if (__any_sync(FULL, !isfinite(ne0) || !isfinite(ne1)) && lane == 0) atomicOr(p.err, ERRBIT_NONFINITE);
#pragma unroll
    for (int n = 0; n < N; ++n) {
      float d[2][CPL];
      f.leave_one_out(n, d);
      // stage E = (xhat - x) * A_Psi and D, rows g and g + 8, the lane's chunk
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        Es[g * LD + CPL * t + q] = ne0 * f.a[n][0][q];
        Es[(g + 8) * LD + CPL * t + q] = ne1 * f.a[n][1][q];
        Ds[g * LD + CPL * t + q] = d[0][q];
        Ds[(g + 8) * LD + CPL * t + q] = d[1][q];
      }
      __syncwarp();
      float part[SL];
      GradTile<K, MATH>::run(Es, Ds, part, lane);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < SL; ++q) {
        const int o = (n * SL + q) * 32 + lane;
        float s = acc_s[o], c = acc_c[o];
        neumaier_add(s, c, part[q]);
        acc_s[o] = s;
        acc_c[o] = c;
      }
    }
  }
  __syncthreads();
  // CTA combine in warp order; partial layout [cta][n][K][K] of (sum, comp)
  const int nw = blockDim.x >> 5;
  float *out = p.partial + size_t(blockIdx.x) * 2 * N * K * K;
  for (int f = threadIdx.x; f < N * SL * 32; f += blockDim.x) {
    float s = 0.f, c = 0.f;
    for (int w = 0; w < nw; ++w) {
      const float *ws = smem + N * TW + w * (L::STAGE + L::ACC) + L::STAGE;
      neumaier_add(s, c, ws[f]);
      c += ws[N * SL * 32 + f];
    }
    const int ln = f & 31, q = (f >> 5) % SL, n = f / (SL * 32);
    const int gg = ln >> 2, tt = ln & 3;
    const int i = q & 3, u = (q >> 2) % (K / 8), mt = (q >> 2) / (K / 8);
    const int j = 16 * mt + gg + 8 * (i >> 1), r = 8 * u + 2 * tt + (i & 1);
    const size_t o = (size_t(n) * K + j) * K + r;
    out[2 * o] = s;
    out[2 * o + 1] = c;
  }
}

// ------------------------------------ core phase, CTA-cooperative (BF16)
// The core-gradient pass (Algorithm 5) for BF16, every order and padded rank.
// Since E^(n) = (xhat - x) * A_Psi^(n) (row-wise scaling),
//   G^(n) = E^(n)T D^(n) = A_Psi^(n)T ((xhat - x) * D^(n)),
// so the residual is folded into D and the contraction runs over the raw rows.
// A CTA tile is WARPS warp tiles (WARPS x 16 nonzeros):
//   phase 1  each warp gathers its 16 nonzeros' rows, forms C^(n) = A_Psi B
//            (Prod), xhat and D^(n), and stores A_Psi^(n) and
//            (xhat - x) * D^(n) as BF16 rows in shared memory;
//   phase 2  the N (K/16)^2 output blocks of 16 x 16 (mode n, rows j of
//            G^(n), columns r) are dealt to the warps; each contracts its
//            blocks over the CTA tile's nonzeros (ldmatrix.trans operands,
//            WARPS k-steps of mma.sync m16n8k16, FP32 accumulation) and adds
//            the CTA tile's block into Neumaier (sum, compensation) registers.
// Every output element has exactly one owning warp, so the CTA partial needs
// no combine; fixed grid and tile order make the pass reproducible bit for bit.
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr)
               : "memory");
}

// C = A_Psi B^(n) for a warp's 16 staged BF16 rows (A operand by ldmatrix,
// natural contraction order), accumulators in the row-chunk layout of
// Prod: y[h][q] is row g + 8h, column r = (K/4) t + q.  The B table holds,
// per n-tile u and k-step s, the lane's (b0, b1) = B rows 16s + 2t (+1) and
// 16s + 2t + 8 (+9) of the output column out_col(u, g) (zero outside
// J_n x R).  The same BF16 roundings as Prod<K, MATH_BF16>.
template <int K>
struct CoopProd {
  static constexpr int NT = K / 8;
  static constexpr int KS = K / 16;
  static constexpr int WORDS = NT * KS * 32 * 2;
  __device__ static void fill(float *tabf, const float *__restrict__ Bn, int J, int R) {
    uint32_t *tab = reinterpret_cast<uint32_t *>(tabf);
    for (int e = threadIdx.x; e < NT * KS * 32; e += blockDim.x) {
      const int lane = e & 31, us = e >> 5, s = us % KS, u = us / KS;
      const int g = lane >> 2, t = lane & 3;
      const int col = out_col<K>(u, g);
      const int k0 = 16 * s + 2 * t;
      tab[2 * e] = pack_bf16(core_entry(Bn, J, R, 0, k0, col), core_entry(Bn, J, R, 0, k0 + 1, col));
      tab[2 * e + 1] = pack_bf16(core_entry(Bn, J, R, 0, k0 + 8, col), core_entry(Bn, J, R, 0, k0 + 9, col));
    }
  }
  // rows_s: shared address of the warp's first staged row; ldb: row stride
  __device__ static void run(uint32_t rows_s, int ldb, const float *tabf, float (&y)[2][K / 4], int lane) {
    const uint2 *tab = reinterpret_cast<const uint2 *>(tabf);
    const int ri = lane & 7, q = lane >> 3;
    uint32_t a[KS][4];
#pragma unroll
    for (int s = 0; s < KS; ++s)
      ldsm_x4(rows_s + (ri + 8 * (q & 1)) * ldb + 2 * (16 * s + 8 * (q >> 1)), a[s][0], a[s][1], a[s][2],
              a[s][3]);
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int s = 0; s < KS; ++s) {
        const uint2 b = tab[(u * KS + s) * 32 + lane];
        mma_bf16(acc, a[s][0], a[s][1], a[s][2], a[s][3], b.x, b.y);
      }
      y[0][2 * u] = acc[0]; y[0][2 * u + 1] = acc[1];
      y[1][2 * u] = acc[2]; y[1][2 * u + 1] = acc[3];
    }
  }
};

template <int N, int K>
struct CoopSmem {
  // 4-warp CTAs (64-nonzero tiles, six per SM) at K = 16, N <= 3: shorter
  // barriers, measured 1% faster than 8-warp CTAs.  16 warps at K = 32,
  // N = 4: one output block per warp (16 blocks), so each warp keeps one
  // block's compensated sums, which brings the pass to 128 registers and
  // 16 warps per SM (measured 25.6 -> 22.1 ms on the order-4 tensor; 12
  // warps: 22.9 ms).  8 warps elsewhere.
  static constexpr int WARPS = (K == 16 && N <= 3) ? 4 : (K == 32 && N == 4) ? 16 : 8;
  static constexpr int ROWS = WARPS * FT_TILE;              // nonzeros per CTA tile
  static constexpr int LDB = 2 * K + 16;                    // bytes per staged row (conflict-free ldmatrix)
  static constexpr int BUF = ROWS * LDB;                    // bytes of one [ROWS][K] bf16 buffer
  static constexpr int TW = CoopProd<K>::WORDS;             // == Prod<K, MATH_BF16>::WORDS
  static constexpr int TAB = N * TW * 4;                    // a.B operand tables
  static constexpr int UNITS = N * (K / 16) * (K / 16);     // 16 x 16 output blocks
  static constexpr int UPW = (UNITS + WARPS - 1) / WARPS;   // blocks per warp
  // A_SMEM: form C = A_Psi B from the staged BF16 rows (ldmatrix) instead of
  // the gathered registers.  It frees the registers that let two CTAs share
  // an SM at (K, N) = (16, 6) and (32, 3); elsewhere it measured 3-4% slower.
  static constexpr bool A_SMEM = (K == 16 && N == 6) || (K == 32 && N == 3);
  // CTAs per SM (the launch bound caps the registers to fit them): six
  // 4-warp CTAs at K = 16, N <= 3 (79 registers, no spills), two up to N = 6
  // and at K = 32, N = 3, else one
  static constexpr int MINB = (K == 16 && N <= 3) ? 6 : ((K == 16 && N <= 6) || (K == 32 && N == 3)) ? 2 : 1;
  static constexpr size_t bytes() { return size_t(TAB) + size_t(2) * N * BUF; }
};

__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                              uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr)
               : "memory");
}

template <int CPL>
__device__ __forceinline__ void coop_store(unsigned char *dst, const uint32_t (&v)[CPL / 2]) {
  if constexpr (CPL == 8) *reinterpret_cast<uint4 *>(dst) = make_uint4(v[0], v[1], v[2], v[3]);
  else *reinterpret_cast<uint2 *>(dst) = make_uint2(v[0], v[1]);
}

// STORE: the storage scheme (rows of C read from p.cst, Sec. 5.6).
// ROWS16: the rows come from the BF16 copies p.abf (half the bytes of the
// float32 rows); otherwise the float32 rows are gathered and rounded here, to
// the same values.
template <int N, int K, bool STORE = false, bool ROWS16 = false>
__global__ void __launch_bounds__(32 * CoopSmem<N, K>::WARPS, CoopSmem<N, K>::MINB) k_core_coop(const EpochArgs p) {
  using L = CoopSmem<N, K>;
  static_assert(CoopProd<K>::WORDS == Prod<K, MATH_BF16>::WORDS, "one table size for both C paths");
  constexpr int CPL = K / 4;
  constexpr int TW = L::TW;
  extern __shared__ __align__(16) float smem[];
  unsigned char *bytes = reinterpret_cast<unsigned char *>(smem);
  unsigned char *abuf = bytes + L::TAB;                     // [N][ROWS] rows of A_Psi^(n)
  unsigned char *dbuf = abuf + N * L::BUF;                  // [N][ROWS] rows of (xhat - x) D^(n)
  const uint32_t abuf_s = static_cast<uint32_t>(__cvta_generic_to_shared(abuf));
  const uint32_t dbuf_s = static_cast<uint32_t>(__cvta_generic_to_shared(dbuf));
  if constexpr (L::A_SMEM) {
#pragma unroll 1
    for (int n = 0; n < N; ++n) CoopProd<K>::fill(smem + n * TW, p.B[n], p.J[n], p.R);
  } else {
    fill_tables<N, K, MATH_BF16>(smem, p, false);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;

  float gs[L::UPW][8], gc[L::UPW][8];
#pragma unroll
  for (int u = 0; u < L::UPW; ++u)
#pragma unroll
    for (int i = 0; i < 8; ++i) gs[u][i] = gc[u][i] = 0.f;
  __syncthreads();

  const int64_t ntiles = (p.end - p.begin + FT_TILE - 1) / FT_TILE;
  const int64_t nct = (ntiles + L::WARPS - 1) / L::WARPS;
  TileCoords<N> cur, nxt;
  if (blockIdx.x < nct) cur.load(p, p.begin + (int64_t(blockIdx.x) * L::WARPS + w) * FT_TILE, lane, true);
  for (int64_t c = blockIdx.x; c < nct; c += gridDim.x) {
    const int64_t cn = c + gridDim.x;
    if (cn < nct) nxt.load(p, p.begin + (cn * L::WARPS + w) * FT_TILE, lane, true);
    // phase 1: this warp's 16 nonzeros (masked ones leave zero rows)
    {
      Front<N, K, MATH_BF16, true> f;
      f.gather(p, cur, lane, nullptr, !ROWS16);
      // the raw rows go to shared memory as BF16 right away (the operand of
      // both products)
      uint32_t av[N][2][CPL / 2];
#pragma unroll
      for (int n = 0; n < N; ++n)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if constexpr (ROWS16) {
            load_chunk_bf16<K>(p.abf[n], f.row[n][h], t, f.valid[h], av[n][h]);
          } else {
#pragma unroll
            for (int q = 0; q < CPL / 2; ++q) av[n][h][q] = pack_bf16(f.a[n][h][2 * q], f.a[n][h][2 * q + 1]);
          }
          coop_store<CPL>(abuf + n * L::BUF + (FT_TILE * w + g + 8 * h) * L::LDB + 2 * CPL * t, av[n][h]);
        }
      if constexpr (STORE) {
        f.load_stored(p, lane);
      } else if constexpr (L::A_SMEM) {
        __syncwarp();
#pragma unroll
        for (int n = 0; n < N; ++n)
          CoopProd<K>::run(abuf_s + n * L::BUF + FT_TILE * w * L::LDB, L::LDB, smem + n * TW, f.c[n], lane);
        f.predict();
      } else {
#pragma unroll
        for (int n = 0; n < N; ++n) Prod<K, MATH_BF16>::run_packed(av[n], smem + n * TW, f.c[n], lane);
        f.predict();
      }
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
          uint32_t dv[CPL / 2];
#pragma unroll
          for (int q = 0; q < CPL / 2; ++q) dv[q] = pack_bf16(ne[h] * d[h][2 * q], ne[h] * d[h][2 * q + 1]);
          coop_store<CPL>(dbuf + n * L::BUF + (FT_TILE * w + g + 8 * h) * L::LDB + 2 * CPL * t, dv);
        }
      }
    }
    __syncthreads();
    // phase 2: this warp's output blocks over the CTA tile's nonzeros
#pragma unroll
    for (int u = 0; u < L::UPW; ++u) {
      const int unit = w + L::WARPS * u;
      if (unit < L::UNITS) {
        const int n = unit / ((K / 16) * (K / 16));
        const int mt = (unit / (K / 16)) % (K / 16), np = unit % (K / 16);
        // ldmatrix.x4.trans: lanes 8q .. 8q + 7 address the 8 rows (nonzeros)
        // of matrix q.  A operand (A_Psi^T, M = j, K = nonzeros): matrix q
        // covers nonzeros 8 (q >> 1) + 0..7 and columns j = 16 mt + 8 (q & 1)
        // + 0..7.  B operand ((xhat - x) D, K = nonzeros, N = r): matrix q
        // covers nonzeros 8 (q & 1) + 0..7 and r = 16 np + 8 (q >> 1) + 0..7,
        // i.e. (b0, b1) of the n-tile 16 np and (b0, b1) of 16 np + 8.
        const int ri = lane & 7, mi = lane >> 3;
        const uint32_t a_addr = abuf_s + n * L::BUF + (ri + 8 * (mi >> 1)) * L::LDB + 2 * (16 * mt + 8 * (mi & 1));
        const uint32_t d_addr = dbuf_s + n * L::BUF + (ri + 8 * (mi & 1)) * L::LDB + 2 * (16 * np + 8 * (mi >> 1));
        float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int kk = 0; kk < L::ROWS / 16; ++kk) {
          uint32_t a0, a1, a2, a3, b0, b1, b2, b3;
          ldsm_x4_trans(a_addr + kk * 16 * L::LDB, a0, a1, a2, a3);
          ldsm_x4_trans(d_addr + kk * 16 * L::LDB, b0, b1, b2, b3);
          mma_bf16(acc[0], a0, a1, a2, a3, b0, b1);
          mma_bf16(acc[1], a0, a1, a2, a3, b2, b3);
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int i = 0; i < 4; ++i) neumaier_add(gs[u][4 * nt + i], gc[u][4 * nt + i], acc[nt][i]);
      }
    }
    __syncthreads();
    cur = nxt;
  }
  // CTA partial in the [n][K][K] layout of (sum, compensation) pairs; every
  // element is written by its owning warp (zero when the CTA had no tiles)
  float *out = p.partial + size_t(blockIdx.x) * 2 * N * K * K;
#pragma unroll
  for (int u = 0; u < L::UPW; ++u) {
    const int unit = w + L::WARPS * u;
    if (unit < L::UNITS) {
      const int n = unit / ((K / 16) * (K / 16));
      const int mt = (unit / (K / 16)) % (K / 16), np = unit % (K / 16);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int j = 16 * mt + g + 8 * (i >> 1), r = 16 * np + 8 * nt + 2 * t + (i & 1);
          const size_t o = (size_t(n) * K + j) * K + r;
          out[2 * o] = gs[u][4 * nt + i];
          out[2 * o + 1] = gc[u][4 * nt + i];
        }
    }
  }
}

// ----------------------------------------------------- predict and errors
// FP32-accurate predictions (three-pass TF32 products; the precision of the
// epochs does not apply here).  MODE 0: write xhat; MODE 1: per-CTA float64
// sums of e^2 and |e|.
template <int N, int K, int MODE>
__global__ void __launch_bounds__(256) k_eval(const EpochArgs p) {
  extern __shared__ __align__(16) float smem[];
  constexpr int TW = Prod<K, MATH_TF32X3>::WORDS;
  fill_tables<N, K, MATH_TF32X3>(smem, p, false);
  __shared__ double red[2][8];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t ntiles = (p.end - p.begin + FT_TILE - 1) / FT_TILE;
  double se = 0.0, ae = 0.0;
  // the next tile's coordinates and values are loaded before the current
  // tile's rows, so the stream's DRAM latency overlaps the gathers
  TileCoords<N> cur, nxt;
  if (warp < ntiles) cur.load(p, p.begin + warp * FT_TILE, lane, MODE == 1);
  for (int64_t tile = warp; tile < ntiles; tile += nwarps) {
    const int64_t next = tile + nwarps;
    if (next < ntiles) nxt.load(p, p.begin + next * FT_TILE, lane, MODE == 1);
    Front<N, K, MATH_TF32X3, true> f;
    f.gather(p, cur, lane);
    cur = nxt;
    f.compute(smem, TW, lane);
    if ((lane & 3) == 0) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!f.valid[h]) continue;
        if constexpr (MODE == 0) {
          p.pred[f.m[h] - p.begin] = f.xhat[h];
        } else {
          const float e = f.x[h] - f.xhat[h];
          if (!isfinite(e)) atomicOr(p.err, ERRBIT_NONFINITE);
          se += double(e) * double(e);
          ae += fabs(double(e));
        }
      }
    }
  }
  if constexpr (MODE == 1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      se += __shfl_xor_sync(FULL, se, o);
      ae += __shfl_xor_sync(FULL, ae, o);
    }
    const int w = threadIdx.x >> 5;
    if (lane == 0) { red[0][w] = se; red[1][w] = ae; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += red[0][i]; b += red[1][i]; }
      p.err_partial[2 * blockIdx.x] = a;
      p.err_partial[2 * blockIdx.x + 1] = b;
    }
  }
}

}  // namespace ft

// ===================================================== batched persistent epoch
// Many independent tensors in one launch per kernel class (N, K, precision).
// The tiles of every tensor of the class are cut into units of a fixed number
// of warp tiles, dealt round-robin over the class's tensors; CTA b takes units
// b, b + G, b + 2G, ...  A CTA reloads the tensor's arguments and operand
// tables when its next unit belongs to another tensor.  The factor pass is
// Hogwild within each tensor; the core pass writes one compensated partial
// per unit, which k_batch_finalize reduces per tensor in a fixed order
// (reproducible bit for bit).
namespace ft {

struct BatchUnit {
  int32_t tensor;       // index into the tensor table
  int32_t pad;
  int64_t tile_begin;   // warp tiles [tile_begin, tile_end) of that tensor
  int64_t tile_end;
  int64_t poff;         // float offset of the unit's core partial (2 * N * K * K floats)
};

struct BatchArgs {
  const EpochArgs *tensors;   // per-tensor arguments (device)
  const BatchUnit *units;     // units of this kernel class
  int nunits;
  float *partial;             // core partials
  const float *hyper;         // lr_a, lambda_a, lr_b, lambda_b (device)
};

// 384-thread CTAs at K = 16 (12 warps per SM at up to 168 registers; 1.6%
// faster than 256 threads on the 64-tensor FP32 epoch), 256 at K = 32
template <int K>
struct BatchFactorLaunch {
  static constexpr int THREADS = (K == 16) ? 384 : 256;
};

template <int N, int K, int MATH>
__global__ void __launch_bounds__(BatchFactorLaunch<K>::THREADS) k_batch_factor(const BatchArgs b) {
  extern __shared__ __align__(16) float smem[];
  __shared__ EpochArgs ea;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  int cur = -1;
  for (int u = blockIdx.x; u < b.nunits; u += gridDim.x) {
    const BatchUnit un = b.units[u];
    if (un.tensor != cur) {
      __syncthreads();
      if (threadIdx.x == 0) {
        ea = b.tensors[un.tensor];
        ea.lr = b.hyper[0];
        ea.lam = b.hyper[1];
      }
      __syncthreads();
      fill_tables<N, K, MATH>(smem, ea, true);
      __syncthreads();
      cur = un.tensor;
    }
    // the branch-free tile (without a cache) where every mode's rows are read
    // as 16-byte groups (full width or narrower than K; one variant for both
    // keeps the registers of the persistent kernel down)
    const bool groups = ea.vec4mask == (1u << N) - 1u;
    for (int64_t tile = un.tile_begin + wid; tile < un.tile_end; tile += wpc) {
      TileCoords<N> tc;
      tc.load(ea, ea.begin + tile * FT_TILE, lane, true);
      if (groups) factor_tile_fast<N, K, MATH, true>(ea, smem, nullptr, nullptr, tc, lane);
      else factor_tile<N, K, MATH, false>(ea, smem, nullptr, nullptr, tc, lane);
    }
  }
}

template <int N, int K, int MATH>
__global__ void __launch_bounds__(256) k_batch_core(const BatchArgs b) {
  extern __shared__ __align__(16) float smem[];
  __shared__ EpochArgs ea;
  using L = CoreSmem<N, K, MATH>;
  constexpr int CPL = K / 4;
  constexpr int TW = L::TW;
  constexpr int LD = L::LD;
  constexpr int SL = GradTile<K, MATH>::SLOTS;
  const int wid = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  float *stage = smem + N * TW + wid * (L::STAGE + L::ACC);
  float *Es = stage, *Ds = stage + FT_TILE * LD;
  float *acc_s = stage + L::STAGE;
  float *acc_c = acc_s + N * SL * 32;
  int cur = -1;
  for (int u = blockIdx.x; u < b.nunits; u += gridDim.x) {
    const BatchUnit un = b.units[u];
    __syncthreads();
    if (un.tensor != cur) {
      if (threadIdx.x == 0) ea = b.tensors[un.tensor];
      __syncthreads();
      fill_tables<N, K, MATH>(smem, ea, false);
      cur = un.tensor;
    }
    for (int q = lane; q < N * SL * 32; q += 32) { acc_s[q] = 0.f; acc_c[q] = 0.f; }
    __syncthreads();
    for (int64_t tile = un.tile_begin + wid; tile < un.tile_end; tile += wpc) {
      Front<N, K, MATH, true> f;
      f.load(ea, ea.begin + tile * FT_TILE, lane, true);
      f.compute(smem, TW, lane);
      const float ne0 = f.xhat[0] - f.x[0], ne1 = f.xhat[1] - f.x[1];
#pragma unroll
      for (int n = 0; n < N; ++n) {
        float d[2][CPL];
        f.leave_one_out(n, d);
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
          Es[g * LD + CPL * t + q] = ne0 * f.a[n][0][q];
          Es[(g + 8) * LD + CPL * t + q] = ne1 * f.a[n][1][q];
          Ds[g * LD + CPL * t + q] = d[0][q];
          Ds[(g + 8) * LD + CPL * t + q] = d[1][q];
        }
        __syncwarp();
        float part[SL];
        GradTile<K, MATH>::run(Es, Ds, part, lane);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < SL; ++q) {
          const int o = (n * SL + q) * 32 + lane;
          float s = acc_s[o], c = acc_c[o];
          neumaier_add(s, c, part[q]);
          acc_s[o] = s;
          acc_c[o] = c;
        }
      }
    }
    __syncthreads();
    float *out = b.partial + un.poff;
    for (int f = threadIdx.x; f < N * SL * 32; f += blockDim.x) {
      float s = 0.f, c = 0.f;
      for (int w = 0; w < wpc; ++w) {
        const float *ws = smem + N * TW + w * (L::STAGE + L::ACC) + L::STAGE;
        neumaier_add(s, c, ws[f]);
        c += ws[N * SL * 32 + f];
      }
      const int ln = f & 31, q = (f >> 5) % SL, n = f / (SL * 32);
      const int gg = ln >> 2, tt = ln & 3;
      const int i = q & 3, uu = (q >> 2) % (K / 8), mt = (q >> 2) / (K / 8);
      const int j = 16 * mt + gg + 8 * (i >> 1), r = 8 * uu + 2 * tt + (i & 1);
      const size_t o = (size_t(n) * K + j) * K + r;
      out[2 * o] = s;
      out[2 * o + 1] = c;
    }
  }
}

}  // namespace ft

// ======================================================== per-row statistics
// Inputs of the learned step size: for every row of every mode, the number of
// nonzeros, the residual sum and the full row gradient
//   g_r = sum_m (-e_m p_m + lambda a_r),  p_m = d_m B^(n)T   (Eq. "Gradient_low_rank_cp")
// (PASS 1), and the curvature along g_r, sum_m (p_m . g_r)^2 (PASS 2),
// accumulated with float atomics.  FP32 on the CUDA cores.
namespace ft {

struct RowStatArgs {
  EpochArgs p;
  float *gsum;                 // row gradients, mode n at goff[n] (I_n x J_n)
  float *cnt, *esum, *hsum;    // per row (rows of all modes concatenated)
  int64_t roff[FT_MAXN];
  int64_t goff[FT_MAXN];
};

template <int N, int K, int PASS>
__global__ void __launch_bounds__(256) k_row_stats(const RowStatArgs s) {
  extern __shared__ __align__(16) float smem[];
  constexpr int CPL = K / 4;
  constexpr int TW = Prod<K, MATH_FP32>::WORDS;
  const EpochArgs &p = s.p;
  fill_tables<N, K, MATH_FP32>(smem, p, true);
  __syncthreads();
  const int lane = threadIdx.x & 31, t = lane & 3;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t ntiles = (p.end - p.begin + FT_TILE - 1) / FT_TILE;
  for (int64_t tile = warp; tile < ntiles; tile += nwarps) {
    Front<N, K, MATH_FP32, true> f;
    f.load(p, p.begin + tile * FT_TILE, lane, true);
    f.compute(smem, TW, lane);
    const float e[2] = {f.x[0] - f.xhat[0], f.x[1] - f.xhat[1]};
#pragma unroll
    for (int n = 0; n < N; ++n) {
      float d[2][CPL], pp[2][CPL];
      f.leave_one_out(n, d);
      Prod<K, MATH_FP32>::run(d, smem + (N + n) * TW, pp, lane);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t row = f.row[n][h];
        float *g = s.gsum + s.goff[n] + row * p.J[n] + CPL * t;
        if constexpr (PASS == 1) {
          if (f.valid[h]) {
#pragma unroll
            for (int q = 0; q < CPL; ++q)
              if (CPL * t + q < p.J[n]) atomicAdd(g + q, fmaf(-e[h], pp[h][q], p.lam * f.a[n][h][q]));
            if (t == 0) {
              atomicAdd(s.cnt + s.roff[n] + row, 1.f);
              atomicAdd(s.esum + s.roff[n] + row, e[h]);
            }
          }
        } else {
          float q2 = 0.f;
          if (f.valid[h]) {
#pragma unroll
            for (int q = 0; q < CPL; ++q)
              if (CPL * t + q < p.J[n]) q2 = fmaf(pp[h][q], g[q], q2);
          }
          q2 += __shfl_xor_sync(FULL, q2, 1);
          q2 += __shfl_xor_sync(FULL, q2, 2);
          if (t == 0 && f.valid[h]) atomicAdd(s.hsum + s.roff[n] + row, q2 * q2);
        }
      }
    }
  }
}

}  // namespace ft
