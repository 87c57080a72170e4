// C ABI of the FastTuckerPlus library (declared in include/ft.h) and the small
// kernels around the epochs: input validation, the deterministic per-row
// reduction, the core finalize step and the float64 error reduction.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <new>
#include <vector>

#include "ft.h"
#include "ft_device.cuh"
#include "ft_internal.h"

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxCoreBlocksPerSm = 8;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// ---------------------------------------------------------------- kernels
struct ValidateArgs {
  const int32_t *idx[FT_MAXN];
  int64_t I[FT_MAXN];
  int N;
  const float *vals;
  int64_t nnz;
  int *err;
};

// Every coordinate in [0, I_n) and every value finite (ft_init).
__global__ void k_validate(const ValidateArgs v) {
  int bad = 0;
  for (int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; m < v.nnz;
       m += int64_t(gridDim.x) * blockDim.x) {
    for (int n = 0; n < v.N; ++n) {
      const int32_t i = v.idx[n][m];
      if (i < 0 || i >= v.I[n]) bad |= ft::ERRBIT_INDEX;
    }
    if (!isfinite(v.vals[m])) bad |= ft::ERRBIT_VALUE;
  }
  bad = __reduce_or_sync(ft::FULL, bad);
  if (bad && (threadIdx.x & 31) == 0) atomicOr(v.err, bad);
}

struct ApplyArgs {
  float *A[FT_MAXN];
  const float *scale[FT_MAXN];
  const int32_t *order[FT_MAXN];
  const int32_t *segptr[FT_MAXN];
  const int32_t *segrow[FT_MAXN];
  int J[FT_MAXN];
  int offJ[FT_MAXN];
  int64_t seg_lo[FT_MAXN];
  int64_t thread_off[FT_MAXN + 1];  // prefix sums of nseg_n * J_n
  int N;
  int sumJ;
  const float *delta;
  float lr;
};

// Deterministic scatter of one batch: for every (mode, row touched in the
// batch, column) the per-nonzero steps are summed in increasing nonzero
// order, then a <- a + lr * s_row * sum (batch-synchronous reading of
// Eq. "Update_FastTuckerPlus_factor").
__global__ void k_apply(const ApplyArgs a) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (tid >= a.thread_off[a.N]) return;
  int n = 0;
  while (tid >= a.thread_off[n + 1]) ++n;
  const int64_t local = tid - a.thread_off[n];
  const int64_t seg = a.seg_lo[n] + local / a.J[n];
  const int j = int(local % a.J[n]);
  const int32_t p0 = a.segptr[n][seg], p1 = a.segptr[n][seg + 1];
  float acc = 0.f;
  for (int32_t q = p0; q < p1; ++q) acc += a.delta[int64_t(a.order[n][q]) * a.sumJ + a.offJ[n] + j];
  const int64_t row = a.segrow[n][seg];
  const float lr = a.scale[n] ? a.lr * a.scale[n][row] : a.lr;
  float *dst = a.A[n] + row * a.J[n] + j;
  *dst = fmaf(lr, acc, *dst);
}

struct FinalizeArgs {
  const float *partial;  // [nparts][N][K][K] of (sum, comp)
  int nparts;
  int N, K, R;
  int J[FT_MAXN];
  int offG[FT_MAXN];
  float *B[FT_MAXN];
  float *G_out;
  float lr, lam;
  float inv_nnz;
  int update;
};

// Core finalize (Algorithm 5): G^(n) = sum over CTA partials (compensated,
// fixed order); B <- B - lr (G / |Omega| + lam B).
// Storage scheme of the core phase (Sec. 5.6): C^(n) = A^(n) B^(n) for every
// row of every mode, FP32, row-major I_n x K with zeros in columns >= R.
// Thread e computes four columns of one row (summing over j in order).
struct StoreArgs {
  const float *A[FT_MAXN];
  const float *B[FT_MAXN];
  float *C[FT_MAXN];
  int64_t I[FT_MAXN];
  int J[FT_MAXN];
  int64_t chunk_begin[FT_MAXN + 1];   // first 4-column chunk of each mode
  int N, K, R;
};

__global__ void k_store_c(const StoreArgs a) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= a.chunk_begin[a.N]) return;
  int n = 0;
  while (n + 1 < a.N && e >= a.chunk_begin[n + 1]) ++n;
  const int64_t local = e - a.chunk_begin[n];
  const int64_t row = local / (a.K / 4);
  const int r0 = 4 * int(local % (a.K / 4));
  const float *arow = a.A[n] + row * a.J[n];
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int j = 0; j < a.J[n]; ++j) {
    const float av = __ldg(arow + j);
    const float *brow = a.B[n] + int64_t(j) * a.R;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (r0 + q < a.R) acc[q] = fmaf(av, __ldg(brow + r0 + q), acc[q]);
  }
  *reinterpret_cast<float4 *>(a.C[n] + row * a.K + r0) = make_float4(acc[0], acc[1], acc[2], acc[3]);
}

// One warp per element of G: lane l sums the partials of CTAs l, l + 32,
// ... in order (Neumaier), then the lanes are combined by a fixed xor tree
// and lane 0 holds the result - the same order on every run.
__global__ void k_finalize(const FinalizeArgs f) {
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int KK = f.K * f.K;
  if (warp >= int64_t(f.N) * KK) return;
  const int e = int(warp);
  const int n = e / KK, j = (e % KK) / f.K, r = e % f.K;
  if (j >= f.J[n] || r >= f.R) return;
  float s = 0.f, c = 0.f;
#pragma unroll 4
  for (int q = lane; q < f.nparts; q += 32) {
    const float2 pp = *reinterpret_cast<const float2 *>(f.partial + (size_t(q) * f.N * KK + e) * 2);
    ft::neumaier_add(s, c, pp.x);
    c += pp.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
    ft::neumaier_add(s, c, s2);
    c += c2;
  }
  if (lane != 0) return;
  const float G = s + c;
  if (f.G_out) f.G_out[f.offG[n] + j * f.R + r] = G;
  if (f.update) {
    float *b = f.B[n] + j * f.R + r;
    const float bv = *b;
    *b = bv - f.lr * fmaf(G, f.inv_nnz, f.lam * bv);
  }
}

struct ErrFinalArgs {
  const double *part;
  int nparts;
  int64_t n;
  double *out3;
};

// Fixed-order float64 reduction of the per-CTA error sums.
__global__ void k_errors_final(const ErrFinalArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double se = 0.0, ae = 0.0;
  for (int q = 0; q < a.nparts; ++q) { se += a.part[2 * q]; ae += a.part[2 * q + 1]; }
  a.out3[0] = a.n > 0 ? sqrt(se / double(a.n)) : 0.0;
  a.out3[1] = a.n > 0 ? ae / double(a.n) : 0.0;
  a.out3[2] = se;
}

struct CountArgs {
  const int32_t *idx[FT_MAXN];
  int32_t *counts[FT_MAXN];
  int N;
  int64_t nnz;
};

// Training nonzeros per row of every mode (selects the cached hot rows).
__global__ void k_row_counts(const CountArgs a) {
  for (int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; m < a.nnz;
       m += int64_t(gridDim.x) * blockDim.x)
    for (int n = 0; n < a.N; ++n) atomicAdd(a.counts[n] + a.idx[n][m], 1);
}

struct RemapArgs {
  const int32_t *idx[FT_MAXN];
  int32_t *out[FT_MAXN];
  const int32_t *slot_of[FT_MAXN];
  int64_t I[FT_MAXN];
  int N;
  int64_t nnz;
  int vec;            // every idx[n] and out[n] 16-byte aligned: 4 coordinates per access
};

__device__ __forceinline__ int32_t remap_one(const RemapArgs &a, int n, int32_t v) {
  const int32_t sl = (v >= 0 && int64_t(v) < a.I[n]) ? __ldg(a.slot_of[n] + v) : -1;
  return sl >= 0 ? -(sl + 1) : v;
}

// Coordinates of the Hogwild pass: a cached row becomes -(slot + 1).  A
// coordinate outside [0, I_n) is passed through unchanged (the epoch kernels
// mask it and latch FT_ERR_INDEX).
__global__ void k_remap(const RemapArgs a) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int64_t n4 = a.vec ? a.nnz / 4 : 0;
  for (int64_t q = tid; q < n4; q += stride)
    for (int n = 0; n < a.N; ++n) {
      const int4 v = __ldcs(reinterpret_cast<const int4 *>(a.idx[n]) + q);
      __stcs(reinterpret_cast<int4 *>(a.out[n]) + q,
             make_int4(remap_one(a, n, v.x), remap_one(a, n, v.y), remap_one(a, n, v.z), remap_one(a, n, v.w)));
    }
  for (int64_t m = 4 * n4 + tid; m < a.nnz; m += stride)
    for (int n = 0; n < a.N; ++n) a.out[n][m] = remap_one(a, n, a.idx[n][m]);
}

// Reordered copy of the nonzeros: out[n][m] = idx[n][perm[m]],
// vals_out[m] = vals[perm[m]].  An entry of perm outside [0, nnz) latches
// ERRBIT_INDEX and copies nonzero 0 instead (the arrays stay valid).
struct PermuteArgs {
  const int32_t *idx[FT_MAXN];
  int32_t *out[FT_MAXN];
  const float *vals;
  float *vals_out;
  const int32_t *perm;
  int N;
  int64_t nnz;
  int *err;
};

// Each thread takes PERMUTE_U positions per round (strided by the grid, so
// every access to perm and to the outputs stays coalesced) and issues all of
// their random gathers before any store, to keep many loads in flight.
constexpr int PERMUTE_U = 4;

__global__ void k_permute(const PermuteArgs a) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t m0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; m0 < a.nnz; m0 += PERMUTE_U * stride) {
    int64_t q[PERMUTE_U];
    bool bad = false;
#pragma unroll
    for (int u = 0; u < PERMUTE_U; ++u) {
      const int64_t m = m0 + u * stride;
      q[u] = m < a.nnz ? int64_t(__ldcs(a.perm + m)) : 0;
      if (q[u] < 0 || q[u] >= a.nnz) {
        bad = bad || m < a.nnz;
        q[u] = 0;
      }
    }
    if (bad) atomicOr(a.err, ft::ERRBIT_INDEX);
    float v[PERMUTE_U];
#pragma unroll
    for (int u = 0; u < PERMUTE_U; ++u) v[u] = __ldg(a.vals + q[u]);
#pragma unroll
    for (int u = 0; u < PERMUTE_U; ++u)
      if (m0 + u * stride < a.nnz) __stcs(a.vals_out + m0 + u * stride, v[u]);
    for (int n = 0; n < a.N; ++n) {
      int32_t c[PERMUTE_U];
#pragma unroll
      for (int u = 0; u < PERMUTE_U; ++u) c[u] = __ldg(a.idx[n] + q[u]);
#pragma unroll
      for (int u = 0; u < PERMUTE_U; ++u)
        if (m0 + u * stride < a.nnz) __stcs(a.out[n] + m0 + u * stride, c[u]);
    }
  }
}

struct RowFinishArgs {
  const float *gsum, *cnt, *esum, *hsum;
  int N;
  int J[FT_MAXN];
  int64_t roff[FT_MAXN + 1];
  int64_t goff[FT_MAXN];
  float lambda, gamma, beta;
  float *ema;      // nullable, in/out
  float *feat;     // rows x 3
  float *label;    // nullable
};

// Features and labels of every row from the accumulated statistics:
// f0 = log(1 + count), f1 = log(1 + ema of |g| / count), f2 = mean residual;
// label = log of the exact line-search step along -g of the row's subproblem,
// shared among the N rows that every nonzero moves at once (divided by N),
// over the step size, clipped to [1/16, 16] (0 for rows without nonzeros).
__global__ void k_row_finish(const RowFinishArgs a) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= a.roff[a.N]) return;
  int n = 0;
  while (q >= a.roff[n + 1]) ++n;
  const int64_t row = q - a.roff[n];
  const float *g = a.gsum + a.goff[n] + row * a.J[n];
  float gg = 0.f;
  for (int j = 0; j < a.J[n]; ++j) gg = fmaf(g[j], g[j], gg);
  const float k = a.cnt[q];
  const float gnorm = sqrtf(gg) / fmaxf(k, 1.f);
  const float ema = a.ema ? a.beta * a.ema[q] + (1.f - a.beta) * gnorm : gnorm;
  if (a.ema) a.ema[q] = ema;
  a.feat[3 * q + 0] = log1pf(k);
  a.feat[3 * q + 1] = log1pf(ema);
  a.feat[3 * q + 2] = k > 0.f ? a.esum[q] / k : 0.f;
  if (a.label) {
    float sc = 1.f;
    const float den = a.hsum[q] + a.lambda * k * gg;
    if (k > 0.f && gg > 0.f && den > 0.f) sc = fminf(fmaxf(gg / den / (float(a.N) * a.gamma), 1.f / 16.f), 16.f);
    a.label[q] = logf(sc);
  }
}

// ------------------------------------------------------------------- plan
struct Plan {
  int N = 0, R = 0, K = 0, sumJ = 0;
  int J[FT_MAXN] = {0};
  int offJ[FT_MAXN] = {0};
  int64_t I[FT_MAXN] = {0};
  int64_t nnz = 0;
  ft_config cfg{};
  int dev = 0, num_sms = 0;
  ft::KernelSet ks;
  ft::EvalSet es;
  int grid_factor = 0, grid_core = 0, grid_eval = 0;
  int grid_factor_tc = 0;            // tcgen05 factor pass (engine FT_ENGINE_TCGEN05)
  int factor_threads = 256;          // CTA of the Hogwild warp-tile pass
  int grid_delta = 0;                // deterministic per-nonzero steps (256-thread CTAs)
  int64_t det_S = 0, nbatches = 0;
  int hot_cap = 0;                   // cache slots, all modes (0 = no cache)
  size_t factor_smem = 0;            // Hogwild pass, tables + cache
  // workspace offsets
  size_t off_err = 0, off_out = 0, off_partial = 0, off_errpart = 0, off_delta = 0;
  size_t off_order = 0, off_segptr = 0, off_segrow = 0;
  size_t off_remap = 0, off_hot = 0, off_counts = 0, off_stats = 0, off_cst = 0, total = 0;
  size_t off_abf = 0;                // BF16 row copies of the BF16 core pass (0 = none)
  size_t off_snap = 0;               // per-CTA snapshots of the hot-row cache
  size_t off_hotw = 0;               // write-back weight of every cache slot
  size_t remap_bytes = 0;            // one of the two remapped coordinate copies
  int64_t rows = 0, grows = 0;      // sum I_n and sum I_n J_n
  // core-gradient kernel of the configured scheme (calculation or storage)
  const void *core_fn = nullptr;
  size_t core_smem = 0;
  int core_threads = 256;
};

// Default shared memory of the hot-row cache per 256 threads of the factor
// CTA: two 256-thread CTAs per SM hold about 100 KB each, one 512-thread CTA
// twice that.
constexpr size_t kHotCacheBytes = 96 * 1024;
constexpr size_t kMaxSmem = 227 * 1024;

ft_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FT_OK : FT_ERR_CUDA; }

// The dynamic shared-memory limit is a property of the kernel function for
// the whole process, so it is only ever raised: a context created later with
// a smaller launch must not lower it under an older context's larger one.
int occupancy(const void *fn, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, size_t> limit;   // (device, kernel)
  int nb = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    size_t &lim = limit[std::make_pair(dev, fn)];
    if (smem > lim) {
      if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
        return 0;
      lim = smem;
    }
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess) return 0;
  return nb;
}

ft_status make_plan(int N, const int64_t *I, const int *J, int R, int64_t nnz, const ft_config *cfg,
                    Plan *p) {
  if (!I || !J || !p) return FT_ERR_ARG;
  if (N < 1 || N > FT_MAX_ORDER) return FT_ERR_SHAPE;
  if (R < 1 || R > FT_MAX_RANK) return FT_ERR_SHAPE;
  if (nnz < 0 || nnz > INT32_MAX) return FT_ERR_ARG;
  ft_config c;
  ft_config_default(&c);
  if (cfg) c = *cfg;
  if (c.precision < FT_FP32 || c.precision > FT_BF16) return FT_ERR_ARG;
  if (c.scatter != FT_HOGWILD && c.scatter != FT_DETERMINISTIC) return FT_ERR_ARG;
  if (c.scatter == FT_DETERMINISTIC && c.det_batch < 1) return FT_ERR_ARG;
  if (c.blocks_per_sm < 0) return FT_ERR_ARG;
  if (c.hot_rows < -1 || c.hot_window < 1 || c.hot_window > (1 << 20) || c.hot_min_count < 1) return FT_ERR_ARG;
  if (c.reserved[0] != 0) return FT_ERR_ARG;
  if (c.l2_persist != 0 && c.l2_persist != 1) return FT_ERR_ARG;
  if (c.core_scheme != FT_CORE_CALC && c.core_scheme != FT_CORE_STORE) return FT_ERR_ARG;
  if (c.engine != FT_ENGINE_WARP && c.engine != FT_ENGINE_TCGEN05) return FT_ERR_ARG;
  if (c.engine == FT_ENGINE_TCGEN05 && (c.scatter != FT_HOGWILD || c.precision != FT_BF16)) return FT_ERR_ARG;
  int maxr = R;
  p->sumJ = 0;
  for (int n = 0; n < N; ++n) {
    if (J[n] < 1 || J[n] > FT_MAX_RANK) return FT_ERR_SHAPE;
    if (I[n] < 1 || I[n] > INT32_MAX) return FT_ERR_SHAPE;
    maxr = std::max(maxr, J[n]);
    p->J[n] = J[n];
    p->I[n] = I[n];
    p->offJ[n] = p->sumJ;
    p->sumJ += J[n];
  }
  const int K = maxr <= 16 ? 16 : 32;
  if (N * K > 160) return FT_ERR_SHAPE;
  p->N = N;
  p->R = R;
  p->K = K;
  p->nnz = nnz;
  p->cfg = c;
  bool ok = ft_kernel_set(N, K, c.precision, &p->ks);
  if (!ok) return FT_ERR_SHAPE;
  ok = K == 16 ? ft_eval_16(N, &p->es) : ft_eval_32(N, &p->es);
  if (!ok) return FT_ERR_SHAPE;

  if (cudaGetDevice(&p->dev) != cudaSuccess) return FT_ERR_CUDA;
  if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->dev) != cudaSuccess)
    return FT_ERR_CUDA;
  int64_t maxI = 1;
  for (int n = 0; n < N; ++n) maxI = std::max(maxI, I[n]);
  const bool tc = c.engine == FT_ENGINE_TCGEN05;
  if (tc && (K != 16 || p->ks.factor_tc == nullptr)) return FT_ERR_ARG;
  const size_t factor_base_smem = tc ? p->ks.factor_tc_smem : p->ks.factor_smem;
  p->hot_cap = 0;
  // The tcgen05 pass with every row full width stages the next tile's rows
  // in shared memory after the cache (4 warpgroups x N x 128 rows of 64 B);
  // the default cache takes what is left.
  bool full_width = true;
  for (int n = 0; n < N; ++n) full_width = full_width && J[n] == K;
  size_t stage_bytes = 0;
  if (c.scatter == FT_HOGWILD && c.hot_rows != 0 && nnz > 0) {
    if (tc && full_width) stage_bytes = size_t(4) * N * 128 * 64;
    const size_t per_slot = size_t(K) * sizeof(float) + 1;
    int64_t sumI = 0;
    for (int n = 0; n < N; ++n) sumI += I[n];
    if (!tc) p->factor_threads = p->ks.factor_threads;
    const size_t budget = tc ? kHotCacheBytes : kHotCacheBytes * size_t(p->factor_threads / 256);
    const int64_t fit = int64_t((kMaxSmem - factor_base_smem - stage_bytes - 64) / per_slot);
    int64_t cap = c.hot_rows > 0 ? c.hot_rows : std::min<int64_t>(int64_t(budget / per_slot), fit);
    cap = std::min(cap, sumI);
    if (cap > fit) return FT_ERR_ARG;
    p->hot_cap = int(std::max<int64_t>(cap, 0));
  }
  p->factor_smem = factor_base_smem + size_t(p->hot_cap) * K * sizeof(float) +
                   ((size_t(p->hot_cap) + 15) / 16) * 16 + stage_bytes;
  (void)maxI;
  if (tc) {
    // one CTA of 4 warpgroups per SM; the CTAs an SM can hold must not ask
    // for more than its 512 TMEM columns (tcgen05.alloc would wait)
    // (checked at the smallest launch, without the cache, where most fit)
    const int occ_max = occupancy(p->ks.factor_tc, p->ks.factor_tc_threads, p->ks.factor_tc_smem);
    const int occ_t = std::min(occupancy(p->ks.factor_tc, p->ks.factor_tc_threads, p->factor_smem),
                               occupancy(p->ks.factor_tc_async, p->ks.factor_tc_threads, p->factor_smem));
    const int per_sm = std::min(occ_t, c.blocks_per_sm ? c.blocks_per_sm : 1);
    if (occ_t < 1 || occ_max * p->ks.factor_tc_tmem_cols > 512) return FT_ERR_CUDA;
    p->grid_factor_tc = p->num_sms * per_sm;
  }
  // without the cache the warp-tile pass runs 256-thread CTAs
  if (p->hot_cap == 0) p->factor_threads = 256;
  const int ft_threads = tc ? 256 : p->factor_threads;
  const int occ_f = std::min({occupancy(p->ks.factor, ft_threads, tc ? p->ks.factor_smem : p->factor_smem),
                              occupancy(p->ks.factor_fast, ft_threads, tc ? p->ks.factor_smem : p->factor_smem),
                              occupancy(p->ks.factor_fast_narrow, ft_threads,
                                        tc ? p->ks.factor_smem : p->factor_smem)});
  const int occ_d = occupancy(p->ks.factor_delta, 256, p->ks.factor_smem);
  const bool store = c.core_scheme == FT_CORE_STORE;
  p->core_fn = store ? p->ks.core_store : p->ks.core;
  p->core_smem = store ? p->ks.core_store_smem : p->ks.core_smem;
  p->core_threads = store ? p->ks.core_store_threads : p->ks.core_threads;
  const int occ_c = occupancy(p->core_fn, p->core_threads, p->core_smem);
  const int occ_p = occupancy(p->es.predict, 256, p->es.smem);
  const int occ_e = occupancy(p->es.errors, 256, p->es.smem);
  if (occ_f < 1 || occ_d < 1 || occ_c < 1 || occ_p < 1 || occ_e < 1) return FT_ERR_CUDA;
  const int bps = c.blocks_per_sm;
  p->grid_factor = p->num_sms * (bps ? bps : occ_f);
  p->grid_delta = p->num_sms * (bps ? bps : occ_d);
  p->grid_core = p->num_sms * std::min(bps ? bps : occ_c, kMaxCoreBlocksPerSm);
  p->grid_eval = p->num_sms * std::min(occ_p, occ_e);

  size_t off = 0;
  p->off_err = off;     off += align_up(sizeof(int) * 16);
  p->off_out = off;     off += align_up(sizeof(double) * 4);
  p->off_partial = off; off += align_up(sizeof(float) * 2 * size_t(p->grid_core) * N * K * K);
  p->off_errpart = off; off += align_up(sizeof(double) * 2 * size_t(p->grid_eval));
  if (p->hot_cap > 0) {
    int64_t sumI = 0;
    for (int n = 0; n < N; ++n) sumI += I[n];
    // two copies: ft_rebind fills the idle one while epochs still read the other
    p->remap_bytes = align_up(sizeof(int32_t) * size_t(N) * nnz);
    p->off_remap = off;  off += 2 * p->remap_bytes;
    p->off_hot = off;    off += align_up(sizeof(int32_t) * size_t(p->hot_cap));
    p->off_counts = off; off += align_up(sizeof(int32_t) * size_t(sumI));
    const int snap_ctas = std::max(p->grid_factor, p->grid_factor_tc);
    p->off_snap = off;   off += align_up(sizeof(float) * size_t(snap_ctas) * p->hot_cap * K);
    p->off_hotw = off;   off += align_up(sizeof(float) * size_t(p->hot_cap));
  }
  if (c.scatter == FT_DETERMINISTIC) {
    p->det_S = std::max<int64_t>(1, std::min<int64_t>(c.det_batch, std::max<int64_t>(nnz, 1)));
    p->nbatches = nnz > 0 ? (nnz + p->det_S - 1) / p->det_S : 0;
    p->off_delta = off;  off += align_up(sizeof(float) * size_t(p->det_S) * p->sumJ);
    p->off_order = off;  off += align_up(sizeof(int32_t) * size_t(N) * nnz);
    p->off_segptr = off; off += align_up(sizeof(int32_t) * size_t(N) * (nnz + 1));
    p->off_segrow = off; off += align_up(sizeof(int32_t) * size_t(N) * std::max<int64_t>(nnz, 1));
  }
  p->rows = 0;
  p->grows = 0;
  for (int n = 0; n < N; ++n) {
    p->rows += I[n];
    p->grows += I[n] * J[n];
  }
  p->off_stats = off; off += align_up(sizeof(float) * size_t(p->grows + 3 * p->rows));
  if (store) {
    p->off_cst = off; off += align_up(sizeof(float) * size_t(p->rows) * K);
  }
  if (c.precision == FT_BF16) {
    p->off_abf = off; off += align_up(sizeof(uint16_t) * size_t(p->rows) * K);
  }
  p->total = off;
  return FT_OK;
}

}  // namespace

// ------------------------------------------------------------------ context
struct ft_ctx {
  Plan p;
  const int32_t *idx[FT_MAXN] = {nullptr};
  const float *vals = nullptr;
  float *A[FT_MAXN] = {nullptr};
  float *B[FT_MAXN] = {nullptr};
  char *ws = nullptr;
  unsigned vecmask = 0;
  unsigned vec4mask = 0;
  std::vector<int64_t> seg_lo[FT_MAXN];  // per mode: first segment of each batch (+ end)
  int hot_base[FT_MAXN + 1] = {0};       // cache slots of mode n: [base[n], base[n+1])
  bool hot_active = false;
  int remap_cur = 0;                     // which remapped copy the Hogwild pass reads
  int64_t launches = 0;
  // l2_persist: the access-policy window over the factor matrices that every
  // launch of this context carries
  bool l2_on = false;
  cudaAccessPolicyWindow l2_window{};
};

namespace {

template <typename T>
T *ws_ptr(ft_ctx *c, size_t off) {
  return reinterpret_cast<T *>(c->ws + off);
}

ft_status launch(ft_ctx *c, const void *fn, int grid, int threads, size_t smem, void *args,
                 cudaStream_t st) {
  if (grid <= 0) return FT_OK;
  void *argv[] = {args};
  cudaError_t e;
  if (c->l2_on) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(threads);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[0].val.accessPolicyWindow = c->l2_window;
    lc.attrs = attr;
    lc.numAttrs = 1;
    e = cudaLaunchKernelExC(&lc, fn, argv);
  } else {
    e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), argv, smem, st);
  }
  ++c->launches;
  return cuda_status(e);
}

// The l2_persist window: the address span of the factor matrices (clamped to
// the device's largest window), marked persisting in L2 for this context's
// launches.  The context's persisting-L2 limit is raised to the window (or
// the device maximum) if it is lower; the hit ratio scales the window down
// to what the limit holds.  Devices without persisting L2 leave it off.
ft_status setup_l2_window(ft_ctx *c) {
  const Plan &p = c->p;
  uintptr_t lo = UINTPTR_MAX, hi = 0;
  for (int n = 0; n < p.N; ++n) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(c->A[n]);
    lo = std::min(lo, a);
    hi = std::max(hi, a + uintptr_t(p.I[n]) * uintptr_t(p.J[n]) * sizeof(float));
  }
  int max_win = 0, max_persist = 0;
  if (cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, p.dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, p.dev) != cudaSuccess)
    return FT_ERR_CUDA;
  if (max_win <= 0 || max_persist <= 0 || hi <= lo) return FT_OK;
  const size_t bytes = std::min<size_t>(hi - lo, size_t(max_win));
  const size_t want = std::min<size_t>(bytes, size_t(max_persist));
  size_t cur = 0;
  if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess) return FT_ERR_CUDA;
  if (cur < want) {
    if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) return FT_ERR_CUDA;
    cur = want;
  }
  c->l2_window.base_ptr = reinterpret_cast<void *>(lo);
  c->l2_window.num_bytes = bytes;
  c->l2_window.hitRatio = float(std::min(1.0, double(cur) / double(bytes)));
  c->l2_window.hitProp = cudaAccessPropertyPersisting;
  c->l2_window.missProp = cudaAccessPropertyStreaming;
  c->l2_on = true;
  return FT_OK;
}

ft::EpochArgs base_args(ft_ctx *c) {
  ft::EpochArgs a;
  memset(&a, 0, sizeof(a));
  for (int n = 0; n < c->p.N; ++n) {
    a.idx[n] = c->idx[n];
    a.A[n] = c->A[n];
    a.B[n] = c->B[n];
    a.I[n] = c->p.I[n];
    a.J[n] = c->p.J[n];
    a.offJ[n] = c->p.offJ[n];
  }
  a.R = c->p.R;
  a.sumJ = c->p.sumJ;
  a.vecmask = c->vecmask;
  a.vec4mask = c->vec4mask;
  a.vals = c->vals;
  a.begin = 0;
  a.end = c->p.nnz;
  a.err = ws_ptr<int>(c, c->p.off_err);
  return a;
}

// Host construction of the deterministic row grouping: for every batch and
// mode, the batch's positions sorted by (row, position) and cut into one
// segment per distinct row.
ft_status build_segments(ft_ctx *c, cudaStream_t st) {
  const Plan &p = c->p;
  const int64_t nnz = p.nnz, S = p.det_S;
  std::vector<int32_t> host_idx(size_t(std::max<int64_t>(nnz, 1)));
  std::vector<int32_t> order(size_t(std::max<int64_t>(nnz, 1)));
  std::vector<int32_t> segptr, segrow;
  std::vector<uint64_t> keys(size_t(std::min<int64_t>(S, std::max<int64_t>(nnz, 1))));
  for (int n = 0; n < p.N; ++n) {
    if (nnz > 0 && cudaMemcpyAsync(host_idx.data(), c->idx[n], sizeof(int32_t) * nnz,
                                   cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return FT_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FT_ERR_CUDA;
    segptr.clear();
    segrow.clear();
    c->seg_lo[n].assign(size_t(p.nbatches + 1), 0);
    for (int64_t b = 0; b < p.nbatches; ++b) {
      const int64_t lo = b * S, hi = std::min(nnz, lo + S);
      c->seg_lo[n][b] = int64_t(segrow.size());
      for (int64_t m = lo; m < hi; ++m)
        keys[size_t(m - lo)] = (uint64_t(uint32_t(host_idx[m])) << 32) | uint64_t(m - lo);
      std::sort(keys.begin(), keys.begin() + (hi - lo));
      int64_t prev = -1;
      for (int64_t k = 0; k < hi - lo; ++k) {
        const int64_t row = int64_t(keys[k] >> 32);
        order[size_t(lo + k)] = int32_t(keys[k] & 0xffffffffu);
        if (row != prev) {
          segptr.push_back(int32_t(lo + k));
          segrow.push_back(int32_t(row));
          prev = row;
        }
      }
    }
    c->seg_lo[n][p.nbatches] = int64_t(segrow.size());
    segptr.push_back(int32_t(nnz));
    int32_t *d_order = ws_ptr<int32_t>(c, p.off_order) + size_t(n) * nnz;
    int32_t *d_segptr = ws_ptr<int32_t>(c, p.off_segptr) + size_t(n) * (nnz + 1);
    int32_t *d_segrow = ws_ptr<int32_t>(c, p.off_segrow) + size_t(n) * std::max<int64_t>(nnz, 1);
    if (nnz > 0 && cudaMemcpyAsync(d_order, order.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st) !=
                       cudaSuccess)
      return FT_ERR_CUDA;
    if (cudaMemcpyAsync(d_segptr, segptr.data(), sizeof(int32_t) * segptr.size(), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return FT_ERR_CUDA;
    if (!segrow.empty() && cudaMemcpyAsync(d_segrow, segrow.data(), sizeof(int32_t) * segrow.size(),
                                           cudaMemcpyHostToDevice, st) != cudaSuccess)
      return FT_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FT_ERR_CUDA;
  }
  return FT_OK;
}

// The Hogwild pass's copy of the coordinates with cached rows remapped to
// -(slot + 1), written into remapped copy `target` (0 or 1); the slot of each
// row (or -1) sits in the counts region.
ft_status remap_hot(ft_ctx *c, cudaStream_t st, int target) {
  const Plan &p = c->p;
  RemapArgs ra;
  memset(&ra, 0, sizeof(ra));
  int64_t off = 0;
  for (int n = 0; n < p.N; ++n) {
    ra.idx[n] = c->idx[n];
    ra.out[n] = ws_ptr<int32_t>(c, p.off_remap + size_t(target) * p.remap_bytes) + size_t(n) * p.nnz;
    ra.slot_of[n] = ws_ptr<int32_t>(c, p.off_counts) + off;
    ra.I[n] = p.I[n];
    off += p.I[n];
  }
  ra.N = p.N;
  ra.nnz = p.nnz;
  ra.vec = 1;
  for (int n = 0; n < p.N; ++n)
    if ((reinterpret_cast<uintptr_t>(ra.idx[n]) | reinterpret_cast<uintptr_t>(ra.out[n])) % 16 != 0) ra.vec = 0;
  const int grid = int(std::min<int64_t>((p.nnz + 1023) / 1024, int64_t(p.num_sms) * 8));
  return launch(c, reinterpret_cast<const void *>(&k_remap), std::max(grid, 1), 256, 0, &ra, st);
}

// Hot-row cache of the Hogwild pass: count the nonzeros of every row, keep
// the hot_cap most frequent rows of each mode that have at least
// hot_min_count of them, and write the remapped coordinates.
ft_status build_hot_cache(ft_ctx *c, cudaStream_t st) {
  const Plan &p = c->p;
  int64_t sumI = 0;
  for (int n = 0; n < p.N; ++n) sumI += p.I[n];
  int32_t *d_counts = ws_ptr<int32_t>(c, p.off_counts);
  if (cudaMemsetAsync(d_counts, 0, sizeof(int32_t) * sumI, st) != cudaSuccess) return FT_ERR_CUDA;
  CountArgs ca;
  memset(&ca, 0, sizeof(ca));
  int64_t off = 0;
  for (int n = 0; n < p.N; ++n) {
    ca.idx[n] = c->idx[n];
    ca.counts[n] = d_counts + off;
    off += p.I[n];
  }
  ca.N = p.N;
  ca.nnz = p.nnz;
  const int grid = int(std::min<int64_t>((p.nnz + 255) / 256, int64_t(p.num_sms) * 8));
  ft_status s = launch(c, reinterpret_cast<const void *>(&k_row_counts), grid, 256, 0, &ca, st);
  if (s != FT_OK) return s;
  std::vector<int32_t> counts(static_cast<size_t>(sumI));
  if (cudaMemcpyAsync(counts.data(), d_counts, sizeof(int32_t) * sumI, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FT_ERR_CUDA;
  std::vector<int32_t> slot_of(size_t(sumI), -1);
  // the hot_cap most frequent rows of the whole tensor (ties: lower mode, then
  // lower row), grouped by mode into contiguous slot ranges
  struct Cand { int32_t count; int32_t n; int32_t r; };
  std::vector<Cand> cand;
  off = 0;
  for (int n = 0; n < p.N; ++n) {
    for (int64_t r = 0; r < p.I[n]; ++r)
      if (counts[size_t(off + r)] >= p.cfg.hot_min_count)
        cand.push_back(Cand{counts[size_t(off + r)], int32_t(n), int32_t(r)});
    off += p.I[n];
  }
  const size_t k = std::min(cand.size(), size_t(p.hot_cap));
  std::partial_sort(cand.begin(), cand.begin() + k, cand.end(), [](const Cand &a, const Cand &b) {
    if (a.count != b.count) return a.count > b.count;
    return a.n != b.n ? a.n < b.n : a.r < b.r;
  });
  cand.resize(k);
  std::sort(cand.begin(), cand.end(), [](const Cand &a, const Cand &b) {
    return a.n != b.n ? a.n < b.n : a.r < b.r;
  });
  // Write-back weight of every slot.  A CTA handles n_w nonzeros between two
  // write-backs (hot_window x 128 nonzeros rounded up to whole CTA tiles, or
  // its whole share of a small tensor).  A row with c of the nnz nonzeros appears x = c n_w /
  // nnz times in that share, and P = G (1 - (1 - c / nnz)^n_w) of the G CTAs
  // are expected to change it between write-backs.  x < 1: the CTAs' changes
  // are distinct steps of distinct nonzeros and add up (w = 1, Hogwild);
  // x >= 1: every CTA moves the row several steps toward the same optimum
  // and the row takes their average (w = 1 / P).
  const int G = p.cfg.engine == FT_ENGINE_TCGEN05 ? p.grid_factor_tc : p.grid_factor;
  const int64_t tile = p.cfg.engine == FT_ENGINE_TCGEN05 ? 512 : 16 * (p.factor_threads / 32);
  const int64_t per_window = (int64_t(p.cfg.hot_window) * 128 + tile - 1) / tile * tile;
  const double n_w = std::min<double>(double(per_window), std::ceil(double(p.nnz) / double(std::max(G, 1))));
  std::vector<float> weight(std::max<size_t>(k, 1), 1.f);
  for (size_t q = 0; q < k; ++q) {
    const double cnt = double(cand[q].count), nnz = double(std::max<int64_t>(p.nnz, 1));
    const double x = cnt * n_w / nnz;
    const double P = double(G) * -std::expm1(n_w * std::log1p(-std::min(cnt / nnz, 1.0 - 1e-12)));
    weight[q] = x >= 1.0 ? float(1.0 / std::max(1.0, P)) : 1.f;
  }
  std::vector<int32_t> hot(std::max<size_t>(k, 1), 0);
  int64_t mode_off[FT_MAXN + 1] = {0};
  for (int n = 0; n < p.N; ++n) mode_off[n + 1] = mode_off[n] + p.I[n];
  for (int n = 0; n <= p.N; ++n) c->hot_base[n] = 0;
  for (size_t q = 0; q < k; ++q) {
    hot[q] = cand[q].r;
    slot_of[size_t(mode_off[cand[q].n] + cand[q].r)] = int32_t(q);
    c->hot_base[cand[q].n + 1] += 1;
  }
  for (int n = 0; n < p.N; ++n) c->hot_base[n + 1] += c->hot_base[n];
  c->hot_active = k > 0;
  if (k == 0) return FT_OK;
  int32_t *d_hot = ws_ptr<int32_t>(c, p.off_hot);
  if (cudaMemcpyAsync(d_hot, hot.data(), sizeof(int32_t) * hot.size(), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(ws_ptr<float>(c, p.off_hotw), weight.data(), sizeof(float) * k, cudaMemcpyHostToDevice,
                      st) != cudaSuccess ||
      cudaMemcpyAsync(d_counts, slot_of.data(), sizeof(int32_t) * sumI, cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    return FT_ERR_CUDA;
  c->remap_cur = 0;
  s = remap_hot(c, st, 0);
  if (s != FT_OK) return s;
  return cudaStreamSynchronize(st) == cudaSuccess ? FT_OK : FT_ERR_CUDA;
}

ft_status take_error(ft_ctx *c, cudaStream_t st) {
  int err = 0;
  int *d = ws_ptr<int>(c, c->p.off_err);
  if (cudaMemcpyAsync(&err, d, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return FT_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FT_ERR_CUDA;
  if (err == 0) return FT_OK;
  if (cudaMemsetAsync(d, 0, sizeof(int), st) != cudaSuccess) return FT_ERR_CUDA;
  if (err & ft::ERRBIT_INDEX) return FT_ERR_INDEX;
  if (err & ft::ERRBIT_TIMEOUT) return FT_ERR_TIMEOUT;
  return FT_ERR_NONFINITE;
}

}  // namespace

// ======================================================================= ABI
extern "C" {

void ft_config_default(ft_config *cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->precision = FT_FP32;
  cfg->scatter = FT_HOGWILD;
  cfg->det_batch = 4096;
  cfg->blocks_per_sm = 0;
  cfg->hot_rows = -1;
  cfg->hot_window = 256;
  cfg->hot_min_count = 2;
}

ft_status ft_workspace_size(int N, const int64_t *I, const int *J, int R, int64_t nnz,
                            const ft_config *cfg, size_t *bytes) {
  if (!bytes) return FT_ERR_ARG;
  Plan p;
  const ft_status s = make_plan(N, I, J, R, nnz, cfg, &p);
  if (s != FT_OK) return s;
  *bytes = p.total;
  return FT_OK;
}

ft_status ft_init(ft_ctx **out, int N, const int64_t *I, const int *J, int R, int64_t nnz,
                  const int32_t *const *idx, const float *vals, float *const *A, float *const *B,
                  void *workspace, size_t ws_bytes, const ft_config *cfg, void *stream) {
  if (!out || !idx || !A || !B || (nnz > 0 && !vals) || !workspace) return FT_ERR_ARG;
  *out = nullptr;
  ft_ctx *c = new (std::nothrow) ft_ctx();
  if (!c) return FT_ERR_ARG;
  ft_status s = make_plan(N, I, J, R, nnz, cfg, &c->p);
  if (s != FT_OK) { delete c; return s; }
  if (ws_bytes < c->p.total || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) {
    delete c;
    return FT_ERR_WORKSPACE;
  }
  for (int n = 0; n < N; ++n) {
    if ((nnz > 0 && !idx[n]) || !A[n] || !B[n]) { delete c; return FT_ERR_ARG; }
    c->idx[n] = idx[n];
    c->A[n] = A[n];
    c->B[n] = B[n];
    // full 16-byte row chunks: rows exactly K wide and a 16-byte aligned base;
    // 16-byte groups of narrower rows: J_n a multiple of 4 and that base
    if (J[n] == c->p.K && (reinterpret_cast<uintptr_t>(A[n]) % 16) == 0) c->vecmask |= 1u << n;
    if (J[n] % 4 == 0 && (reinterpret_cast<uintptr_t>(A[n]) % 16) == 0) c->vec4mask |= 1u << n;
  }
  c->vals = vals;
  c->ws = static_cast<char *>(workspace);
  if (c->p.cfg.l2_persist) {
    s = setup_l2_window(c);
    if (s != FT_OK) { delete c; return s; }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(c->ws, 0, c->p.off_partial, st) != cudaSuccess) { delete c; return FT_ERR_CUDA; }
  if (nnz > 0) {
    ValidateArgs v;
    memset(&v, 0, sizeof(v));
    for (int n = 0; n < N; ++n) { v.idx[n] = idx[n]; v.I[n] = I[n]; }
    v.N = N;
    v.vals = vals;
    v.nnz = nnz;
    v.err = ws_ptr<int>(c, c->p.off_err);
    const int grid = int(std::min<int64_t>((nnz + 255) / 256, int64_t(c->p.num_sms) * 8));
    s = launch(c, reinterpret_cast<const void *>(&k_validate), grid, 256, 0, &v, st);
    if (s != FT_OK) { delete c; return s; }
    int err = 0;
    if (cudaMemcpyAsync(&err, v.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      delete c;
      return FT_ERR_CUDA;
    }
    if (err & ft::ERRBIT_INDEX) { delete c; return FT_ERR_INDEX; }
    if (err & ft::ERRBIT_VALUE) { delete c; return FT_ERR_NONFINITE; }
  }
  if (c->p.cfg.scatter == FT_DETERMINISTIC) {
    s = build_segments(c, st);
    if (s != FT_OK) { delete c; return s; }
  }
  if (c->p.hot_cap > 0) {
    s = build_hot_cache(c, st);
    if (s != FT_OK) { delete c; return s; }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) { delete c; return FT_ERR_CUDA; }
  *out = c;
  return FT_OK;
}

ft_status ft_epoch_factors(ft_ctx *c, float lr_a, float lambda_a, const float *const *row_step_scale,
                           void *stream) {
  if (!c) return FT_ERR_ARG;
  if (!std::isfinite(lr_a) || !std::isfinite(lambda_a)) return FT_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Plan &p = c->p;
  if (p.nnz == 0) return FT_OK;
  ft::EpochArgs a = base_args(c);
  a.lr = lr_a;
  a.lam = lambda_a;
  if (row_step_scale)
    for (int n = 0; n < p.N; ++n) a.scale[n] = row_step_scale[n];
  if (p.cfg.scatter == FT_HOGWILD) {
    if (c->hot_active) {
      for (int n = 0; n < p.N; ++n)
        a.idx[n] = ws_ptr<int32_t>(c, p.off_remap + size_t(c->remap_cur) * p.remap_bytes) + size_t(n) * p.nnz;
      for (int n = 0; n <= p.N; ++n) a.hot_base[n] = c->hot_base[n];
      a.hot_rows = ws_ptr<int32_t>(c, p.off_hot);
      a.hot_cap = p.hot_cap;
      a.hot_window = p.cfg.hot_window;
      a.hot_snap = ws_ptr<float>(c, p.off_snap);
      a.hot_weight = ws_ptr<float>(c, p.off_hotw);
    }
    bool scaled = false;
    for (int n = 0; n < p.N; ++n) scaled = scaled || a.scale[n] != nullptr;
    const bool fast = c->hot_active && !scaled && c->vecmask == (1u << p.N) - 1u;
    if (p.cfg.engine == FT_ENGINE_TCGEN05)
      return launch(c, fast ? p.ks.factor_tc_async : p.ks.factor_tc, p.grid_factor_tc, p.ks.factor_tc_threads,
                    c->hot_active ? p.factor_smem : p.ks.factor_tc_smem, &a, st);
    // rows read as 16-byte groups in every mode, some narrower than K
    const bool narrow = !fast && c->hot_active && !scaled && c->vec4mask == (1u << p.N) - 1u;
    return launch(c, fast ? p.ks.factor_fast : (narrow ? p.ks.factor_fast_narrow : p.ks.factor), p.grid_factor,
                  p.factor_threads, c->hot_active ? p.factor_smem : p.ks.factor_smem, &a, st);
  }

  a.delta = ws_ptr<float>(c, p.off_delta);
  ApplyArgs ap;
  memset(&ap, 0, sizeof(ap));
  ap.N = p.N;
  ap.sumJ = p.sumJ;
  ap.delta = a.delta;
  ap.lr = lr_a;
  for (int n = 0; n < p.N; ++n) {
    ap.A[n] = c->A[n];
    ap.scale[n] = a.scale[n];
    ap.order[n] = ws_ptr<int32_t>(c, p.off_order) + size_t(n) * p.nnz;
    ap.segptr[n] = ws_ptr<int32_t>(c, p.off_segptr) + size_t(n) * (p.nnz + 1);
    ap.segrow[n] = ws_ptr<int32_t>(c, p.off_segrow) + size_t(n) * std::max<int64_t>(p.nnz, 1);
    ap.J[n] = p.J[n];
    ap.offJ[n] = p.offJ[n];
  }
  for (int64_t b = 0; b < p.nbatches; ++b) {
    a.begin = b * p.det_S;
    a.end = std::min(p.nnz, a.begin + p.det_S);
    const int64_t tiles = (a.end - a.begin + FT_TILE - 1) / FT_TILE;
    const int grid = int(std::min<int64_t>(p.grid_delta, (tiles + 7) / 8));
    ft_status s = launch(c, p.ks.factor_delta, grid, 256, p.ks.factor_smem, &a, st);
    if (s != FT_OK) return s;
    ap.thread_off[0] = 0;
    for (int n = 0; n < p.N; ++n) {
      ap.seg_lo[n] = c->seg_lo[n][b];
      const int64_t nseg = c->seg_lo[n][b + 1] - c->seg_lo[n][b];
      ap.thread_off[n + 1] = ap.thread_off[n] + nseg * p.J[n];
    }
    const int64_t nthr = ap.thread_off[p.N];
    s = launch(c, reinterpret_cast<const void *>(&k_apply), int((nthr + 255) / 256), 256, 0, &ap, st);
    if (s != FT_OK) return s;
  }
  return FT_OK;
}

struct RowsBf16Args {
  const float *A[FT_MAXN];
  uint32_t *out[FT_MAXN];       // row-major I_n x K/2 words
  int J[FT_MAXN];
  int64_t wbegin[FT_MAXN + 1];  // first word of mode n over all modes
  int N, K;
};

// BF16 copy of every factor row for the BF16 core pass: row i of mode n
// becomes K values (zeros past J_n), rounded to nearest even exactly as the
// core pass rounds the float32 rows it gathers; one thread per word.
__global__ void k_rows_bf16(const RowsBf16Args a) {
  const int64_t total = a.wbegin[a.N];
  for (int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < total;
       w += int64_t(gridDim.x) * blockDim.x) {
    int n = 0;
    while (n + 1 < a.N && w >= a.wbegin[n + 1]) ++n;
    const int64_t local = w - a.wbegin[n];
    const int64_t row = local / (a.K / 2);
    const int j = 2 * int(local % (a.K / 2));
    const float *src = a.A[n] + row * a.J[n];
    const float lo = j < a.J[n] ? __ldg(src + j) : 0.f;
    const float hi = j + 1 < a.J[n] ? __ldg(src + j + 1) : 0.f;
    a.out[n][local] = ft::pack_bf16(lo, hi);
  }
}

// Core gradient over the nonzeros [lo, hi) and, with update, the step
// B <- B - lr_b (G / (hi - lo) + lambda_b B) (Algorithm 5 on that range).
static ft_status core_pass(ft_ctx *c, float lr_b, float lambda_b, float *G_out, int update,
                           cudaStream_t st, int64_t lo = 0, int64_t hi = -1) {
  const Plan &p = c->p;
  if (hi < 0) hi = p.nnz;
  ft::EpochArgs a = base_args(c);
  a.begin = lo;
  a.end = hi;
  a.partial = ws_ptr<float>(c, p.off_partial);
  ft_status s = FT_OK;
  if (p.cfg.core_scheme == FT_CORE_STORE) {
    // storage scheme: C^(n) = A^(n) B^(n) for every row, then the pass reads it
    StoreArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.N = p.N;
    sa.K = p.K;
    sa.R = p.R;
    int64_t off = 0;
    for (int n = 0; n < p.N; ++n) {
      sa.A[n] = c->A[n];
      sa.B[n] = c->B[n];
      sa.J[n] = p.J[n];
      sa.I[n] = p.I[n];
      sa.C[n] = ws_ptr<float>(c, p.off_cst) + off * p.K;
      a.cst[n] = sa.C[n];
      sa.chunk_begin[n] = off * (p.K / 4);
      off += p.I[n];
    }
    sa.chunk_begin[p.N] = off * (p.K / 4);
    const int64_t chunks = sa.chunk_begin[p.N];
    s = launch(c, reinterpret_cast<const void *>(&k_store_c), int((chunks + 255) / 256), 256, 0, &sa, st);
    if (s != FT_OK) return s;
  }
  if (p.off_abf != 0) {
    // BF16 rows for the cooperative pass, made once per core phase (A does
    // not change during it: later sets of ft_epoch_core_sgd reuse the copy)
    RowsBf16Args ra;
    memset(&ra, 0, sizeof(ra));
    ra.N = p.N;
    ra.K = p.K;
    int64_t w = 0;
    for (int n = 0; n < p.N; ++n) {
      ra.A[n] = c->A[n];
      ra.J[n] = p.J[n];
      ra.out[n] = ws_ptr<uint32_t>(c, p.off_abf) + w;
      ra.wbegin[n] = w;
      a.abf[n] = ra.out[n];
      w += p.I[n] * (p.K / 2);
    }
    ra.wbegin[p.N] = w;
    if (lo == 0) {
      const int grid = int(std::min<int64_t>((w + 255) / 256, int64_t(p.num_sms) * 16));
      s = launch(c, reinterpret_cast<const void *>(&k_rows_bf16), grid, 256, 0, &ra, st);
      if (s != FT_OK) return s;
    }
  }
  s = launch(c, p.core_fn, p.grid_core, p.core_threads, p.core_smem, &a, st);
  if (s != FT_OK) return s;
  FinalizeArgs f;
  memset(&f, 0, sizeof(f));
  f.partial = a.partial;
  f.nparts = p.grid_core;
  f.N = p.N;
  f.K = p.K;
  f.R = p.R;
  int off = 0;
  for (int n = 0; n < p.N; ++n) {
    f.J[n] = p.J[n];
    f.B[n] = c->B[n];
    f.offG[n] = off;
    off += p.J[n] * p.R;
  }
  f.G_out = G_out;
  f.lr = lr_b;
  f.lam = lambda_b;
  f.inv_nnz = hi > lo ? float(1.0 / double(hi - lo)) : 0.f;
  f.update = update;
  const int total = p.N * p.K * p.K;
  return launch(c, reinterpret_cast<const void *>(&k_finalize), (32 * total + 255) / 256, 256, 0, &f, st);
}

ft_status ft_epoch_core(ft_ctx *c, float lr_b, float lambda_b, void *stream) {
  if (!c) return FT_ERR_ARG;
  if (!std::isfinite(lr_b) || !std::isfinite(lambda_b)) return FT_ERR_ARG;
  return core_pass(c, lr_b, lambda_b, nullptr, 1, static_cast<cudaStream_t>(stream));
}

ft_status ft_permute(ft_ctx *c, const int32_t *perm, int32_t *const *idx_out, float *vals_out,
                     void *stream) {
  if (!c) return FT_ERR_ARG;
  const Plan &p = c->p;
  if (p.nnz == 0) return FT_OK;
  if (!perm || !idx_out || !vals_out || vals_out == c->vals) return FT_ERR_ARG;
  for (int n = 0; n < p.N; ++n)
    for (int k = 0; k < p.N; ++k)
      if (!idx_out[n] || idx_out[n] == c->idx[k]) return FT_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PermuteArgs a;
  memset(&a, 0, sizeof(a));
  for (int n = 0; n < p.N; ++n) {
    a.idx[n] = c->idx[n];
    a.out[n] = idx_out[n];
  }
  a.vals = c->vals;
  a.vals_out = vals_out;
  a.perm = perm;
  a.N = p.N;
  a.nnz = p.nnz;
  a.err = ws_ptr<int>(c, p.off_err);
  const int grid = int(std::min<int64_t>((p.nnz + 255) / 256, int64_t(p.num_sms) * 16));
  ft_status s = launch(c, reinterpret_cast<const void *>(&k_permute), grid, 256, 0, &a, st);
  if (s != FT_OK) return s;
  for (int n = 0; n < p.N; ++n) c->idx[n] = idx_out[n];
  c->vals = vals_out;
  if (c->hot_active) {
    s = remap_hot(c, st, 1 - c->remap_cur);
    if (s != FT_OK) return s;
    c->remap_cur = 1 - c->remap_cur;
  }
  if (p.cfg.scatter == FT_DETERMINISTIC) return build_segments(c, st);
  return FT_OK;
}

ft_status ft_rebind(ft_ctx *c, const int32_t *const *idx, const float *vals, void *stream) {
  if (!c) return FT_ERR_ARG;
  const Plan &p = c->p;
  if (p.nnz == 0) return FT_OK;
  if (!idx || !vals) return FT_ERR_ARG;
  for (int n = 0; n < p.N; ++n)
    if (!idx[n]) return FT_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int n = 0; n < p.N; ++n) c->idx[n] = idx[n];
  c->vals = vals;
  if (c->hot_active) {
    // the idle remapped copy: passes enqueued before this call keep reading the
    // other one, so the rebuild may run on another stream while they finish
    const ft_status s = remap_hot(c, st, 1 - c->remap_cur);
    if (s != FT_OK) return s;
    c->remap_cur = 1 - c->remap_cur;
  }
  if (p.cfg.scatter == FT_DETERMINISTIC) return build_segments(c, st);
  return FT_OK;
}

ft_status ft_epoch_core_sgd(ft_ctx *c, float lr_b, float lambda_b, int64_t set_size, void *stream) {
  if (!c || set_size < 1) return FT_ERR_ARG;
  if (!std::isfinite(lr_b) || !std::isfinite(lambda_b)) return FT_ERR_ARG;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int64_t lo = 0; lo < c->p.nnz; lo += set_size) {
    const ft_status s = core_pass(c, lr_b, lambda_b, nullptr, 1, st, lo, std::min(c->p.nnz, lo + set_size));
    if (s != FT_OK) return s;
  }
  return FT_OK;
}

ft_status ft_core_grad(ft_ctx *c, float *G_out, void *stream) {
  if (!c || !G_out) return FT_ERR_ARG;
  return core_pass(c, 0.f, 0.f, G_out, 0, static_cast<cudaStream_t>(stream));
}

struct CoreApplyArgs {
  const float *G;        // sum_n J_n R entries, the layout of ft_core_grad
  float *B[FT_MAXN];
  int offG[FT_MAXN + 1];  // first entry of mode n's block; offG[N] = total
  int N;
  float lr, lam, inv_nnz;
};

// The step of Algorithm 5 from a gradient summed elsewhere (for example over
// the shards of Omega held by several processes): one thread per entry,
// B <- B - lr (G inv_nnz + lam B), the arithmetic of k_finalize's update.
__global__ void k_core_apply(const CoreApplyArgs a) {
  const int e = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= a.offG[a.N]) return;
  int n = 0;
  while (n + 1 < a.N && e >= a.offG[n + 1]) ++n;
  float *b = a.B[n] + (e - a.offG[n]);
  const float bv = *b;
  *b = bv - a.lr * fmaf(__ldg(a.G + e), a.inv_nnz, a.lam * bv);
}

ft_status ft_core_apply(ft_ctx *c, const float *G, int64_t nnz_total, float lr_b, float lambda_b,
                        void *stream) {
  if (!c || !G || nnz_total < 0) return FT_ERR_ARG;
  if (!std::isfinite(lr_b) || !std::isfinite(lambda_b)) return FT_ERR_ARG;
  const Plan &p = c->p;
  CoreApplyArgs a;
  memset(&a, 0, sizeof(a));
  a.G = G;
  a.N = p.N;
  int off = 0;
  for (int n = 0; n < p.N; ++n) {
    a.B[n] = c->B[n];
    a.offG[n] = off;
    off += p.J[n] * p.R;
  }
  a.offG[p.N] = off;
  a.lr = lr_b;
  a.lam = lambda_b;
  a.inv_nnz = nnz_total > 0 ? float(1.0 / double(nnz_total)) : 0.f;
  return launch(c, reinterpret_cast<const void *>(&k_core_apply), (off + 255) / 256, 256, 0, &a,
                static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------- core gradient, no allocation
// Scratch of ft_core_grad_noalloc: a 256-byte error word followed by the
// per-CTA (sum, compensation) partials of the core-gradient kernel.  It is a
// file-scope device array, so every GPU that loads this library holds it
// until the process exits, and every call shares it.
#define FT_NOALLOC_SCRATCH_BYTES (16u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[FT_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_lock;
void *g_noalloc_addr[kNoallocMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
ft_status noalloc_scratch(int dev, void **out) {
  if (dev < 0 || dev >= kNoallocMaxDevices) return FT_ERR_CUDA;
  std::lock_guard<std::mutex> guard(g_noalloc_lock);
  if (g_noalloc_addr[dev] == nullptr) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return FT_ERR_CUDA;
    g_noalloc_addr[dev] = ptr;
  }
  *out = g_noalloc_addr[dev];
  return FT_OK;
}
}  // namespace

ft_status ft_core_grad_noalloc(int N, const int64_t *I, const int *J, int R, int64_t nnz,
                               const int32_t *const *idx, const float *vals, const float *const *A,
                               const float *const *B, int precision, float *G_out, void *stream) {
  if (!I || !J || !G_out || (nnz > 0 && (!idx || !vals)) || !A || !B) return FT_ERR_ARG;
  ft_config cfg;
  ft_config_default(&cfg);
  cfg.precision = precision;
  cfg.hot_rows = 0;
  Plan p;
  ft_status s = make_plan(N, I, J, R, nnz, &cfg, &p);
  if (s != FT_OK) return s;
  const size_t need = 256 + sizeof(float) * 2 * size_t(p.grid_core) * N * p.K * p.K;
  if (need > FT_NOALLOC_SCRATCH_BYTES) return FT_ERR_WORKSPACE;
  void *scratch = nullptr;
  s = noalloc_scratch(p.dev, &scratch);
  if (s != FT_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int *err = static_cast<int *>(scratch);
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return FT_ERR_CUDA;

  ft::EpochArgs a;
  memset(&a, 0, sizeof(a));
  for (int n = 0; n < N; ++n) {
    if ((nnz > 0 && !idx[n]) || !A[n] || !B[n]) return FT_ERR_ARG;
    a.idx[n] = nnz > 0 ? idx[n] : nullptr;
    a.A[n] = const_cast<float *>(A[n]);  // read only in the core pass
    a.B[n] = B[n];
    a.I[n] = I[n];
    a.J[n] = J[n];
    a.offJ[n] = p.offJ[n];
    if (J[n] == p.K && (reinterpret_cast<uintptr_t>(A[n]) % 16) == 0) a.vecmask |= 1u << n;
    if (J[n] % 4 == 0 && (reinterpret_cast<uintptr_t>(A[n]) % 16) == 0) a.vec4mask |= 1u << n;
  }
  a.R = R;
  a.sumJ = p.sumJ;
  a.vals = vals;
  a.begin = 0;
  a.end = nnz;
  a.err = err;
  a.partial = reinterpret_cast<float *>(static_cast<char *>(scratch) + 256);
  // the core pass that gathers float32 rows (no room for BF16 row copies);
  // the same grid and order as the context's pass, so the same result
  if (occupancy(p.ks.core_f32rows, p.ks.core_threads, p.ks.core_smem) < 1) return FT_ERR_CUDA;
  void *argv_core[] = {&a};
  if (cudaLaunchKernel(p.ks.core_f32rows, dim3(p.grid_core), dim3(p.ks.core_threads), argv_core, p.ks.core_smem,
                       st) != cudaSuccess)
    return FT_ERR_CUDA;
  FinalizeArgs f;
  memset(&f, 0, sizeof(f));
  f.partial = a.partial;
  f.nparts = p.grid_core;
  f.N = N;
  f.K = p.K;
  f.R = R;
  int off = 0;
  for (int n = 0; n < N; ++n) {
    f.J[n] = J[n];
    f.offG[n] = off;
    off += J[n] * R;
  }
  f.G_out = G_out;
  f.update = 0;
  void *argv_fin[] = {&f};
  const int total = N * p.K * p.K;
  if (cudaLaunchKernel(reinterpret_cast<const void *>(&k_finalize), dim3((32 * total + 255) / 256), dim3(256), argv_fin,
                       0, st) != cudaSuccess)
    return FT_ERR_CUDA;
  int h_err = 0;
  if (cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FT_ERR_CUDA;
  if (h_err & ft::ERRBIT_INDEX) return FT_ERR_INDEX;
  if (h_err) return FT_ERR_NONFINITE;
  return FT_OK;
}

static ft_status eval_args(ft_ctx *c, int64_t n, const int32_t *const *idx, ft::EpochArgs *a) {
  if (n < 0 || n > INT32_MAX) return FT_ERR_ARG;
  if (n > 0 && !idx) return FT_ERR_ARG;
  *a = base_args(c);
  for (int k = 0; k < c->p.N; ++k) {
    if (n > 0 && !idx[k]) return FT_ERR_ARG;
    a->idx[k] = n > 0 ? idx[k] : nullptr;
  }
  a->begin = 0;
  a->end = n;
  return FT_OK;
}

ft_status ft_predict(ft_ctx *c, int64_t n, const int32_t *const *idx, float *out, void *stream) {
  if (!c || (n > 0 && !out)) return FT_ERR_ARG;
  ft::EpochArgs a;
  ft_status s = eval_args(c, n, idx, &a);
  if (s != FT_OK || n == 0) return s;
  a.pred = out;
  const int64_t tiles = (n + FT_TILE - 1) / FT_TILE;
  const int grid = int(std::min<int64_t>(c->p.grid_eval, (tiles + 7) / 8));
  return launch(c, c->p.es.predict, grid, 256, c->p.es.smem, &a, static_cast<cudaStream_t>(stream));
}

ft_status ft_rmse(ft_ctx *c, int64_t n, const int32_t *const *idx, const float *vals, double *out3,
                  void *stream) {
  if (!c || !out3 || (n > 0 && !vals)) return FT_ERR_ARG;
  ft::EpochArgs a;
  ft_status s = eval_args(c, n, idx, &a);
  if (s != FT_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  a.vals = vals;
  a.err_partial = ws_ptr<double>(c, c->p.off_errpart);
  const int grid = c->p.grid_eval;
  s = launch(c, c->p.es.errors, grid, 256, c->p.es.smem, &a, st);
  if (s != FT_OK) return s;
  ErrFinalArgs fa;
  fa.part = a.err_partial;
  fa.nparts = grid;
  fa.n = n;
  fa.out3 = ws_ptr<double>(c, c->p.off_out);
  s = launch(c, reinterpret_cast<const void *>(&k_errors_final), 1, 32, 0, &fa, st);
  if (s != FT_OK) return s;
  if (cudaMemcpyAsync(out3, fa.out3, sizeof(double) * 3, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return FT_ERR_CUDA;
  return take_error(c, st);
}

ft_status ft_row_stats(ft_ctx *c, float lambda_a, float lr_a, float ema_beta, float *ema, float *features,
                       float *labels, void *stream) {
  if (!c || !features || !(lr_a > 0.f) || !std::isfinite(lambda_a) || !(ema_beta >= 0.f && ema_beta <= 1.f))
    return FT_ERR_ARG;
  const Plan &p = c->p;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float *base = ws_ptr<float>(c, p.off_stats);
  if (cudaMemsetAsync(base, 0, sizeof(float) * size_t(p.grows + 3 * p.rows), st) != cudaSuccess) return FT_ERR_CUDA;
  ft::RowStatArgs s;
  memset(&s, 0, sizeof(s));
  s.p = base_args(c);
  s.p.lam = lambda_a;
  s.gsum = base;
  s.cnt = base + p.grows;
  s.esum = s.cnt + p.rows;
  s.hsum = s.esum + p.rows;
  int64_t ro = 0, go = 0;
  for (int n = 0; n < p.N; ++n) {
    s.roff[n] = ro;
    s.goff[n] = go;
    ro += p.I[n];
    go += p.I[n] * p.J[n];
  }
  const int grid = p.num_sms * 4;
  ft_status st1 = FT_OK;
  if (p.nnz > 0) {
    st1 = launch(c, p.es.row_stats1, grid, 256, p.es.stats_smem, &s, st);
    if (st1 == FT_OK && labels) st1 = launch(c, p.es.row_stats2, grid, 256, p.es.stats_smem, &s, st);
    if (st1 != FT_OK) return st1;
  }
  RowFinishArgs f;
  memset(&f, 0, sizeof(f));
  f.gsum = s.gsum;
  f.cnt = s.cnt;
  f.esum = s.esum;
  f.hsum = s.hsum;
  f.N = p.N;
  for (int n = 0; n < p.N; ++n) {
    f.J[n] = p.J[n];
    f.roff[n] = s.roff[n];
    f.goff[n] = s.goff[n];
  }
  f.roff[p.N] = p.rows;
  f.lambda = lambda_a;
  f.gamma = lr_a;
  f.beta = ema_beta;
  f.ema = ema;
  f.feat = features;
  f.label = labels;
  return launch(c, reinterpret_cast<const void *>(&k_row_finish), int((p.rows + 255) / 256), 256, 0, &f, st);
}

ft_status ft_check(ft_ctx *c, void *stream) {
  if (!c) return FT_ERR_ARG;
  return take_error(c, static_cast<cudaStream_t>(stream));
}

int64_t ft_launch_count(const ft_ctx *c) { return c ? c->launches : 0; }

void ft_destroy(ft_ctx *c) { delete c; }

const char *ft_status_str(ft_status s) {
  switch (s) {
    case FT_OK: return "ok";
    case FT_ERR_ARG: return "invalid argument";
    case FT_ERR_INDEX: return "coordinate out of range";
    case FT_ERR_SHAPE: return "unsupported shape";
    case FT_ERR_CUDA: return "CUDA error";
    case FT_ERR_NONFINITE: return "non-finite value or residual";
    case FT_ERR_TIMEOUT: return "device wait timed out";
    case FT_ERR_WORKSPACE: return "workspace too small or misaligned";
  }
  return "unknown status";
}

}  // extern "C"
