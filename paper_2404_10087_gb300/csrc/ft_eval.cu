// Explicit instantiations of the prediction / error kernels (FP32-accurate
// three-pass TF32 products) and the row-statistics kernels for one
// padded rank K (built with FT_K in {16, 32}).
#include "ft_device.cuh"
#include "ft_internal.h"

#ifndef FT_K
#error "FT_K must be defined (16 or 32)"
#endif

#define FT_CAT_(a, b) a##_##b
#define FT_CAT(a, b) FT_CAT_(a, b)

namespace {
template <int N>
ft::EvalSet make_eval() {
  ft::EvalSet s;
  s.predict = reinterpret_cast<const void *>(&ft::k_eval<N, FT_K, 0>);
  s.errors = reinterpret_cast<const void *>(&ft::k_eval<N, FT_K, 1>);
  s.smem = size_t(N) * ft::Prod<FT_K, ft::MATH_TF32X3>::WORDS * sizeof(float);
  s.row_stats1 = reinterpret_cast<const void *>(&ft::k_row_stats<N, FT_K, 1>);
  s.row_stats2 = reinterpret_cast<const void *>(&ft::k_row_stats<N, FT_K, 2>);
  s.stats_smem = 2 * size_t(N) * ft::Prod<FT_K, ft::MATH_FP32>::WORDS * sizeof(float);
  return s;
}
}  // namespace

bool FT_CAT(ft_eval, FT_K)(int N, ft::EvalSet *out) {
  switch (N) {
    case 1: *out = make_eval<1>(); return true;
    case 2: *out = make_eval<2>(); return true;
    case 3: *out = make_eval<3>(); return true;
    case 4: *out = make_eval<4>(); return true;
    case 5: *out = make_eval<5>(); return true;
#if FT_K == 16
    case 6: *out = make_eval<6>(); return true;
    case 7: *out = make_eval<7>(); return true;
    case 8: *out = make_eval<8>(); return true;
    case 9: *out = make_eval<9>(); return true;
    case 10: *out = make_eval<10>(); return true;
#endif
    default: return false;
  }
}
