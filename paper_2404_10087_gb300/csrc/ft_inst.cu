// Explicit instantiations of the epoch kernels for one padded rank K, one
// precision and one order N.  Built once per (FT_K, FT_MATH, FT_N) so the
// units compile in parallel.
#include "ft_device.cuh"
#include "ft_internal.h"
#if FT_K == 16 && FT_MATH == 2
#include "ft_tc05.cuh"
#endif
#if FT_MATH == 0
#include "ft_core32.cuh"
#endif

#ifndef FT_K
#error "FT_K must be defined (16 or 32)"
#endif
#ifndef FT_MATH
#error "FT_MATH must be defined (0 = FP32, 1 = TF32, 2 = BF16)"
#endif

#ifndef FT_N
#error "FT_N must be defined (the order N of this unit)"
#endif

#define FT_CAT_(a, b, c, d) a##_##b##_##c##_##d
#define FT_CAT(a, b, c, d) FT_CAT_(a, b, c, d)

// Arithmetic of the core-gradient kernels for the precision of this unit:
// FT_FP32 runs them on FP32-accurate three-pass TF32 tensor-core products.
#if FT_MATH == 0
#define FT_KMATH ft::MATH_TF32X3
#else
#define FT_KMATH FT_MATH
#endif

// Arithmetic of the factor kernels: FT_FP32 forms a.B and d.B^T on
// FP32-accurate three-pass TF32 tensor-core products (measured faster than
// the CUDA-core form, which costs K^2 FMAs, K shuffles and K/2 shared loads
// per row and product: 11.1 against 15.6 ms on the Netflix-shaped tensor).
#if FT_MATH == 0
#define FT_FMATH ft::MATH_TF32X3
#else
#define FT_FMATH FT_MATH
#endif

namespace {
template <int N>
ft::KernelSet make_set() {
  ft::KernelSet s;
  s.factor = reinterpret_cast<const void *>(&ft::k_factor<N, FT_K, FT_FMATH, false>);
  s.factor_fast = reinterpret_cast<const void *>(&ft::k_factor<N, FT_K, FT_FMATH, false, true>);
  s.factor_fast_narrow = reinterpret_cast<const void *>(&ft::k_factor<N, FT_K, FT_FMATH, false, true, true>);
  s.factor_delta = reinterpret_cast<const void *>(&ft::k_factor<N, FT_K, FT_FMATH, true>);
  s.core = reinterpret_cast<const void *>(&ft::k_core<N, FT_K, FT_KMATH>);
  s.factor_smem = ft::FactorSmem<N, FT_K, FT_FMATH>::tables();
  s.factor_threads = ft::FactorLaunch<N, FT_K, FT_FMATH>::THREADS;
  s.core_smem = ft::CoreSmem<N, FT_K, FT_KMATH>::bytes();
  s.core_threads = 32 * ft::CoreSmem<N, FT_K, FT_KMATH>::WARPS;
  s.batch_factor = reinterpret_cast<const void *>(&ft::k_batch_factor<N, FT_K, FT_FMATH>);
  s.batch_factor_threads = ft::BatchFactorLaunch<FT_K>::THREADS;
  s.batch_core = reinterpret_cast<const void *>(&ft::k_batch_core<N, FT_K, FT_KMATH>);
  s.batch_core_smem = ft::CoreSmem<N, FT_K, FT_KMATH>::bytes();
  s.batch_core_threads = 32 * ft::CoreSmem<N, FT_K, FT_KMATH>::WARPS;
#if FT_MATH == 2
  s.core_store = reinterpret_cast<const void *>(&ft::k_core_coop<N, FT_K, true, true>);
  s.core_store_smem = ft::CoopSmem<N, FT_K>::bytes();
  s.core_store_threads = 32 * ft::CoopSmem<N, FT_K>::WARPS;
#else
  s.core_store = reinterpret_cast<const void *>(&ft::k_core<N, FT_K, FT_KMATH, true>);
  s.core_store_smem = ft::CoreSmem<N, FT_K, FT_KMATH>::bytes();
  s.core_store_threads = 32 * ft::CoreSmem<N, FT_K, FT_KMATH>::WARPS;
#endif
#if FT_MATH == 0
  // FP32 at K = 16 with N <= 5 and at K = 32 with N <= 4: the CTA-cooperative
  // FP32-accurate core pass
  if constexpr ((FT_K == 16 && N <= 5) || (FT_K == 32 && N <= 4)) {
    s.core = reinterpret_cast<const void *>(&ft::k_core32<N, FT_K>);
    s.core_smem = ft::Core32<N, FT_K>::bytes();
    s.core_threads = 32 * ft::Core32<N, FT_K>::WARPS;
    s.batch_core = reinterpret_cast<const void *>(&ft::k_batch_core32<N, FT_K>);
    s.batch_core_smem = ft::Core32<N, FT_K>::bytes();
    s.batch_core_threads = 32 * ft::Core32<N, FT_K>::WARPS;
  }
#endif
#if FT_MATH == 2
  // BF16: the CTA-cooperative core pass on the BF16 row copies; the caller
  // without a workspace (no room for the copies) gathers the float32 rows
  s.core = reinterpret_cast<const void *>(&ft::k_core_coop<N, FT_K, false, true>);
  s.core_smem = ft::CoopSmem<N, FT_K>::bytes();
  s.core_threads = 32 * ft::CoopSmem<N, FT_K>::WARPS;
  s.core_f32rows = reinterpret_cast<const void *>(&ft::k_core_coop<N, FT_K, false, false>);
#else
  s.core_f32rows = s.core;
#endif
#if FT_K == 16 && FT_MATH == 2
  if constexpr (N <= 4) {
    s.factor_tc = reinterpret_cast<const void *>(&ft::k_factor_tc<N>);
    s.factor_tc_async = reinterpret_cast<const void *>(&ft::k_factor_tc<N, true>);
    s.factor_tc_smem = ft::tc::Smem<N>::bytes(0);
    s.factor_tc_threads = ft::tc::THREADS;
    s.factor_tc_tmem_cols = ft::tc::Smem<N>::TMEM_COLS;
  }
#endif
  return s;
}
}  // namespace

bool FT_CAT(ft_kernels, FT_K, FT_MATH, FT_N)(ft::KernelSet *out) {
  *out = make_set<FT_N>();
  return true;
}
