// Explicit instantiations of the epoch kernels for one padded rank K and one
// precision.  Built once per (FT_K, FT_MATH) pair so the units compile in
// parallel.
#include "ft_device.cuh"
#include "ft_internal.h"

#ifndef FT_K
#error "FT_K must be defined (16 or 32)"
#endif
#ifndef FT_MATH
#error "FT_MATH must be defined (0 = FP32, 1 = TF32, 2 = BF16)"
#endif

#define FT_CAT_(a, b, c) a##_##b##_##c
#define FT_CAT(a, b, c) FT_CAT_(a, b, c)

namespace {
template <int N>
ft::KernelSet make_set() {
  ft::KernelSet s;
  s.factor = reinterpret_cast<const void *>(&ft::k_factor<N, FT_K, FT_MATH, false>);
  s.factor_delta = reinterpret_cast<const void *>(&ft::k_factor<N, FT_K, FT_MATH, true>);
  s.core = reinterpret_cast<const void *>(&ft::k_core<N, FT_K, FT_MATH>);
  s.factor_smem = ft::FactorSmem<N, FT_K, FT_MATH>::tables();
  s.core_smem = ft::CoreSmem<N, FT_K, FT_MATH>::bytes();
  s.core_threads = 32 * ft::CoreSmem<N, FT_K, FT_MATH>::WARPS;
#if FT_K == 16 && FT_MATH == 2
  // BF16 at K = 16: the register-resident core pass (no shared-memory staging)
  if constexpr (N <= 4) {
    s.core = reinterpret_cast<const void *>(&ft::k_core_bf16r<N>);
    s.core_smem = ft::CoreRegSmem<N>::bytes();
    s.core_threads = 256;
  }
#endif
  return s;
}
}  // namespace

bool FT_CAT(ft_kernels, FT_K, FT_MATH)(int N, ft::KernelSet *out) {
  switch (N) {
    case 1: *out = make_set<1>(); return true;
    case 2: *out = make_set<2>(); return true;
    case 3: *out = make_set<3>(); return true;
    case 4: *out = make_set<4>(); return true;
#if FT_K == 16
    case 5: *out = make_set<5>(); return true;
    case 6: *out = make_set<6>(); return true;
    case 7: *out = make_set<7>(); return true;
    case 8: *out = make_set<8>(); return true;
#endif
    default: return false;
  }
}
