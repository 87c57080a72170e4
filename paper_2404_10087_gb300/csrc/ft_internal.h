// Host-side declarations shared by the C ABI and the kernel instantiation
// units.  Not part of the public interface.
#pragma once

#include <cstddef>

namespace ft {

// Kernels of one (N, K, precision) instantiation.
struct KernelSet {
  const void *factor = nullptr;        // Hogwild factor pass
  // the same pass with the hot-row cache, every mode full width and one step
  // size for every row (the tile without data-dependent branches)
  const void *factor_fast = nullptr;
  const void *factor_fast_narrow = nullptr;
  const void *factor_delta = nullptr;  // deterministic factor pass (writes per-nonzero steps)
  const void *core = nullptr;          // core-gradient pass
  // the same pass without the BF16 row copies of the workspace (gathers the
  // float32 rows; equal results); `core` itself at FP32 and TF32
  const void *core_f32rows = nullptr;
  size_t factor_smem = 0;              // tables only; the hot-row cache adds to it
  int factor_threads = 256;            // CTA of the cached Hogwild pass (FactorLaunch)
  size_t core_smem = 0;
  int core_threads = 256;
  // core-gradient pass of the storage scheme (rows of C = A B precomputed)
  const void *core_store = nullptr;
  size_t core_store_smem = 0;
  int core_store_threads = 256;
  // batched persistent kernels of this class (generic core, shared-memory staging)
  const void *batch_factor = nullptr;
  int batch_factor_threads = 256;
  const void *batch_core = nullptr;
  size_t batch_core_smem = 0;
  int batch_core_threads = 256;
  // tcgen05 Hogwild factor pass (BF16, K = 16, N <= 4), or null
  const void *factor_tc = nullptr;
  // the same pass with the rows of the next tile arriving by asynchronous copies
  // (hot-row cache on, every row full width, one step size)
  const void *factor_tc_async = nullptr;
  size_t factor_tc_smem = 0;           // without the hot-row cache
  int factor_tc_threads = 0;
  int factor_tc_tmem_cols = 0;         // TMEM columns one CTA allocates
};

// FP32 prediction / error / row-statistics kernels of one (N, K).
struct EvalSet {
  const void *predict = nullptr;
  const void *errors = nullptr;
  size_t smem = 0;
  const void *row_stats1 = nullptr;   // row gradients, counts, residual sums
  const void *row_stats2 = nullptr;   // curvature along the row gradients
  size_t stats_smem = 0;
};

}  // namespace ft

// One entry point per compiled instantiation unit (ft_inst.cu built with
// FT_K in {16, 32}, FT_MATH in {0, 1, 2} and FT_N in 1..10 at K = 16, 1..5 at
// K = 32; ft_eval.cu built with FT_K).
#define FT_SETS_OF(X, K, M) X(K, M, 1) X(K, M, 2) X(K, M, 3) X(K, M, 4) X(K, M, 5)
#define FT_SETS16(X, M) FT_SETS_OF(X, 16, M) X(16, M, 6) X(16, M, 7) X(16, M, 8) X(16, M, 9) X(16, M, 10)
#define FT_ALL_SETS(X) \
  FT_SETS16(X, 0) FT_SETS16(X, 1) FT_SETS16(X, 2) FT_SETS_OF(X, 32, 0) FT_SETS_OF(X, 32, 1) FT_SETS_OF(X, 32, 2)
#define FT_DECLARE_SET(K, M, N) bool ft_kernels_##K##_##M##_##N(ft::KernelSet *out);
FT_ALL_SETS(FT_DECLARE_SET)
#undef FT_DECLARE_SET

// Kernels of one (N, K, precision), false if that combination is not built.
inline bool ft_kernel_set(int N, int K, int precision, ft::KernelSet *out) {
#define FT_CASE(KK, MM, NN) \
  if (K == KK && precision == MM && N == NN) return ft_kernels_##KK##_##MM##_##NN(out);
  FT_ALL_SETS(FT_CASE)
#undef FT_CASE
  return false;
}

bool ft_eval_16(int N, ft::EvalSet *out);
bool ft_eval_32(int N, ft::EvalSet *out);
