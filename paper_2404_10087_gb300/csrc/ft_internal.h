// Host-side declarations shared by the C ABI and the kernel instantiation
// units.  Not part of the public interface.
#pragma once

#include <cstddef>

namespace ft {

// Kernels of one (N, K, precision) instantiation.
struct KernelSet {
  const void *factor = nullptr;        // Hogwild factor pass
  const void *factor_delta = nullptr;  // deterministic factor pass (writes per-nonzero steps)
  const void *core = nullptr;          // core-gradient pass
  size_t factor_smem = 0;              // tables only; the hot-row cache adds to it
  size_t core_smem = 0;
  int core_threads = 256;
};

// FP32 prediction / error kernels of one (N, K).
struct EvalSet {
  const void *predict = nullptr;
  const void *errors = nullptr;
  size_t smem = 0;
};

}  // namespace ft

// One entry point per compiled instantiation unit (ft_inst.cu built with
// FT_K in {16, 32} and FT_MATH in {0, 1, 2}; ft_eval.cu built with FT_K).
#define FT_DECLARE_SET(K, M) bool ft_kernels_##K##_##M(int N, ft::KernelSet *out);
FT_DECLARE_SET(16, 0)
FT_DECLARE_SET(16, 1)
FT_DECLARE_SET(16, 2)
FT_DECLARE_SET(32, 0)
FT_DECLARE_SET(32, 1)
FT_DECLARE_SET(32, 2)
#undef FT_DECLARE_SET
bool ft_eval_16(int N, ft::EvalSet *out);
bool ft_eval_32(int N, ft::EvalSet *out);
