// Checks the three-pass TF32 split's integer rounding of the library
// (Prod<K, MATH_TF32X3>::round_bits) against the conversion instruction
// cvt.rna.tf32.f32 on every float32 bit pattern that is finite and does not
// round past the float32 maximum.  Prints the counts; exits 1 on any
// difference.
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#include "ft_device.cuh"

namespace {

__device__ __forceinline__ uint32_t cvt_rna(float f) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
  return r;
}

__global__ void k_check(unsigned long long *bad, unsigned long long *checked) {
  unsigned long long nb = 0, nc = 0;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < (1ull << 32);
       i += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t b = uint32_t(i);
    if ((b & 0x7fffffffu) >= 0x7f7ff000u) continue;   // inf, NaN, values rounding past the maximum
    const float f = __uint_as_float(b);
    ++nc;
    if (ft::Prod<16, ft::MATH_TF32X3>::round_bits(f) != cvt_rna(f)) ++nb;
  }
  atomicAdd(bad, nb);
  atomicAdd(checked, nc);
}

}  // namespace

int main() {
  unsigned long long *d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return 2;
  if (cudaMemset(d, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) return 2;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) return 2;
  k_check<<<sms * 8, 256>>>(d, d + 1);
  if (cudaDeviceSynchronize() != cudaSuccess) return 2;
  unsigned long long h[2] = {0, 0};
  if (cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return 2;
  cudaFree(d);
  printf("checked %llu mismatches %llu\n", h[1], h[0]);
  return h[0] == 0 && h[1] > 0 ? 0 : 1;
}
