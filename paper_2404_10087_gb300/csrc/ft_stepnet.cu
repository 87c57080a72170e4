// Step-size network (include/ft.h, "step-size network"): a 3 -> 64 -> 64 -> 1
// MLP that maps row statistics to per-row step multipliers of the factor
// update.  BF16 working weights, FP32 accumulation, FP32 masters with Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "ft.h"

namespace {

constexpr int H = 64;
constexpr int NP = H * 3 + H + H * H + H + H + 1;  // 4481 parameters
constexpr int NPP = (NP + 3) / 4 * 4;              // padded to 16 bytes
constexpr int OFF_W1 = 0, OFF_B1 = H * 3, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H;

// Buffer layout (floats): master | adam m | adam v | gradient | last gradient |
// bf16 copies (NPP halves) | step (int) and loss (double) in the last 16 bytes.
struct NetView {
  float *master, *m, *v, *grad, *last;
  __nv_bfloat16 *w;
  int *step;
  double *loss;
};

__host__ __device__ inline NetView view(void *net) {
  float *f = static_cast<float *>(net);
  NetView nv;
  nv.master = f;
  nv.m = f + NPP;
  nv.v = f + 2 * NPP;
  nv.grad = f + 3 * NPP;
  nv.last = f + 4 * NPP;
  nv.w = reinterpret_cast<__nv_bfloat16 *>(f + 5 * NPP);
  char *tail = reinterpret_cast<char *>(f + 5 * NPP + NPP / 2);
  nv.step = reinterpret_cast<int *>(tail);
  nv.loss = reinterpret_cast<double *>(tail + 8);
  return nv;
}

constexpr size_t kBytes = sizeof(float) * (5 * NPP + NPP / 2) + 16;

__device__ inline uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_net_init(void *net, uint64_t seed) {
  NetView nv = view(net);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NPP; q += gridDim.x * blockDim.x) {
    const float u = float(splitmix64(seed * 0x100000001B3ull + uint64_t(q)) >> 40) * (1.f / 16777216.f);
    float w = 0.f;
    if (q < OFF_B1) w = (2.f * u - 1.f) * sqrtf(6.f / 3.f);
    else if (q >= OFF_W2 && q < OFF_B2) w = (2.f * u - 1.f) * sqrtf(6.f / H);
    else if (q >= OFF_W3 && q < OFF_B3) w = (2.f * u - 1.f) * sqrtf(6.f / H);
    if (q >= NP) w = 0.f;
    nv.master[q] = w;
    nv.m[q] = nv.v[q] = nv.grad[q] = nv.last[q] = 0.f;
    nv.w[q] = __float2bfloat16_rn(w);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *nv.step = 0;
    *nv.loss = 0.0;
  }
}

__device__ inline void load_weights(const NetView &nv, float *W) {
  for (int q = threadIdx.x; q < NP; q += blockDim.x) W[q] = __bfloat162float(nv.w[q]);
  __syncthreads();
}

// Multiplier of the linear output u (a log-multiplier), clamped to [1/16, 16].
constexpr float kLogSMax = 2.772588722239781f;   // log 16
__device__ inline float net_output(float u) { return expf(fminf(fmaxf(u, -kLogSMax), kLogSMax)); }

__global__ void __launch_bounds__(128) k_net_forward(const NetView nv, int64_t rows, const float *feat,
                                                      float *scale) {
  __shared__ float W[NP];
  load_weights(nv, W);
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < rows;
       r += int64_t(gridDim.x) * blockDim.x) {
    const float x0 = feat[3 * r], x1 = feat[3 * r + 1], x2 = feat[3 * r + 2];
    float h1[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const float s = W[OFF_B1 + j] + W[OFF_W1 + 3 * j] * x0 + W[OFF_W1 + 3 * j + 1] * x1 + W[OFF_W1 + 3 * j + 2] * x2;
      h1[j] = fmaxf(s, 0.f);
    }
    float z = W[OFF_B3];
    for (int i = 0; i < H; ++i) {
      float s = W[OFF_B2 + i];
#pragma unroll
      for (int j = 0; j < H; ++j) s = fmaf(W[OFF_W2 + H * i + j], h1[j], s);
      z = fmaf(W[OFF_W3 + i], fmaxf(s, 0.f), z);
    }
    scale[r] = net_output(z);
  }
}

// Gradient of (1/rows) sum 1/2 (u - y)^2 (u the linear output, y the
// log-multiplier label).  One warp per block; each chunk of
// 32 rows (one per lane) leaves its activations in shared memory, then lane l
// accumulates the gradient of columns l and l + 32 over the chunk (lane-private
// shared-memory accumulators for W2), and at the end every lane adds its
// share to the global gradient.
constexpr int LDH = H + 1;
struct BackSmem {
  float W[NP];
  float H1[32 * LDH], H2[32 * LDH], DH2[32 * LDH], DH1[32 * LDH];
  float X[32 * 3], DZ[32];
  float ACC2[H * H];   // [i][j], lane l owns columns l and l + 32
};

__global__ void __launch_bounds__(32) k_net_backward(const NetView nv, int64_t rows, const float *feat,
                                                      const float *label, float inv_n) {
  extern __shared__ __align__(16) float smem_raw[];
  BackSmem &S = *reinterpret_cast<BackSmem *>(smem_raw);
  load_weights(nv, S.W);
  const int l = threadIdx.x;
  for (int q = l; q < H * H; q += 32) S.ACC2[q] = 0.f;
  float gW1[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, gb1[2] = {0.f, 0.f}, gb2[2] = {0.f, 0.f};
  float gw3[2] = {0.f, 0.f}, gb3 = 0.f;
  double loss = 0.0;
  __syncwarp();
  for (int64_t base = int64_t(blockIdx.x) * 32; base < rows; base += int64_t(gridDim.x) * 32) {
    const int64_t r = base + l;
    const bool valid = r < rows;
    const float x0 = valid ? feat[3 * r] : 0.f, x1 = valid ? feat[3 * r + 1] : 0.f;
    const float x2 = valid ? feat[3 * r + 2] : 0.f;
    S.X[3 * l] = x0;
    S.X[3 * l + 1] = x1;
    S.X[3 * l + 2] = x2;
    float h1[H], dh1[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const float s = S.W[OFF_B1 + j] + S.W[OFF_W1 + 3 * j] * x0 + S.W[OFF_W1 + 3 * j + 1] * x1 +
                      S.W[OFF_W1 + 3 * j + 2] * x2;
      h1[j] = fmaxf(s, 0.f);
      S.H1[l * LDH + j] = h1[j];
      dh1[j] = 0.f;
    }
    float z = S.W[OFF_B3];
    for (int i = 0; i < H; ++i) {
      float s = S.W[OFF_B2 + i];
#pragma unroll
      for (int j = 0; j < H; ++j) s = fmaf(S.W[OFF_W2 + H * i + j], h1[j], s);
      const float h2 = fmaxf(s, 0.f);
      S.H2[l * LDH + i] = h2;
      z = fmaf(S.W[OFF_W3 + i], h2, z);
    }
    const float res = valid ? z - label[r] : 0.f;
    loss += 0.5 * double(res) * double(res);
    const float dz = res * inv_n;
    S.DZ[l] = dz;
    for (int i = 0; i < H; ++i) {
      const float dh2 = S.H2[l * LDH + i] > 0.f ? dz * S.W[OFF_W3 + i] : 0.f;
      S.DH2[l * LDH + i] = dh2;
#pragma unroll
      for (int j = 0; j < H; ++j) dh1[j] = fmaf(dh2, S.W[OFF_W2 + H * i + j], dh1[j]);
    }
#pragma unroll
    for (int j = 0; j < H; ++j) S.DH1[l * LDH + j] = h1[j] > 0.f ? dh1[j] : 0.f;
    __syncwarp();
    // column sums over the chunk's 32 rows
    for (int rr = 0; rr < 32; ++rr) {
      const float ha = S.H1[rr * LDH + l], hb = S.H1[rr * LDH + l + 32];
      for (int i = 0; i < H; ++i) {
        const float a = S.DH2[rr * LDH + i];
        S.ACC2[H * i + l] = fmaf(a, ha, S.ACC2[H * i + l]);
        S.ACC2[H * i + l + 32] = fmaf(a, hb, S.ACC2[H * i + l + 32]);
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int col = l + 32 * c;
        const float d1 = S.DH1[rr * LDH + col];
        gb1[c] += d1;
#pragma unroll
        for (int k = 0; k < 3; ++k) gW1[c][k] = fmaf(d1, S.X[3 * rr + k], gW1[c][k]);
        gb2[c] += S.DH2[rr * LDH + col];
        gw3[c] = fmaf(S.DZ[rr], S.H2[rr * LDH + col], gw3[c]);
      }
      if (l == 0) gb3 += S.DZ[rr];
    }
    __syncwarp();
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int col = l + 32 * c;
    for (int k = 0; k < 3; ++k) atomicAdd(nv.grad + OFF_W1 + 3 * col + k, gW1[c][k]);
    atomicAdd(nv.grad + OFF_B1 + col, gb1[c]);
    atomicAdd(nv.grad + OFF_B2 + col, gb2[c]);
    atomicAdd(nv.grad + OFF_W3 + col, gw3[c]);
    for (int i = 0; i < H; ++i) atomicAdd(nv.grad + OFF_W2 + H * i + col, S.ACC2[H * i + col]);
  }
  if (l == 0) atomicAdd(nv.grad + OFF_B3, gb3);
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  if (l == 0) atomicAdd(nv.loss, loss);
}

__global__ void k_net_adam(const NetView nv, float lr) {
  const int t = *nv.step + 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, float(t)), c2 = 1.f - powf(b2, float(t));
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NP; q += gridDim.x * blockDim.x) {
    const float g = nv.grad[q];
    const float m = b1 * nv.m[q] + (1.f - b1) * g;
    const float v = b2 * nv.v[q] + (1.f - b2) * g * g;
    nv.m[q] = m;
    nv.v[q] = v;
    const float w = nv.master[q] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    nv.master[q] = w;
    nv.w[q] = __float2bfloat16_rn(w);
    nv.last[q] = g;
    nv.grad[q] = 0.f;
  }
}

__global__ void k_net_step(const NetView nv) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *nv.step += 1;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

size_t ft_stepnet_bytes(void) { return kBytes; }

ft_status ft_stepnet_init(void *net, uint64_t seed, void *stream) {
  if (!net || !aligned16(net)) return FT_ERR_ARG;
  k_net_init<<<8, 256, 0, static_cast<cudaStream_t>(stream)>>>(net, seed);
  return cudaGetLastError() == cudaSuccess ? FT_OK : FT_ERR_CUDA;
}

ft_status ft_stepnet_forward(const void *net, int64_t rows, const float *features, float *scale, void *stream) {
  if (!net || !aligned16(net) || rows < 0 || (rows > 0 && (!features || !scale))) return FT_ERR_ARG;
  if (rows == 0) return FT_OK;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FT_ERR_CUDA;
  const int64_t blocks = std::min<int64_t>((rows + 127) / 128, int64_t(sms) * 8);
  k_net_forward<<<unsigned(blocks), 128, 0, static_cast<cudaStream_t>(stream)>>>(view(const_cast<void *>(net)), rows,
                                                                                features, scale);
  return cudaGetLastError() == cudaSuccess ? FT_OK : FT_ERR_CUDA;
}

ft_status ft_stepnet_train(void *net, int64_t rows, const float *features, const float *labels, float lr, int steps,
                           double *loss_out, void *stream) {
  if (!net || !aligned16(net) || rows < 1 || !features || !labels || steps < 0 || !(lr >= 0.f))
    return FT_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const NetView nv = view(net);
  const size_t smem = sizeof(BackSmem);
  if (cudaFuncSetAttribute(reinterpret_cast<const void *>(&k_net_backward),
                           cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
    return FT_ERR_CUDA;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FT_ERR_CUDA;
  const int64_t blocks = std::min<int64_t>((rows + 31) / 32, int64_t(sms) * 4);
  for (int s = 0; s < steps; ++s) {
    if (cudaMemsetAsync(nv.loss, 0, sizeof(double), st) != cudaSuccess) return FT_ERR_CUDA;
    k_net_backward<<<unsigned(blocks), 32, smem, st>>>(nv, rows, features, labels, float(1.0 / double(rows)));
    k_net_adam<<<8, 256, 0, st>>>(nv, lr);
    k_net_step<<<1, 32, 0, st>>>(nv);
    if (cudaGetLastError() != cudaSuccess) return FT_ERR_CUDA;
  }
  if (loss_out) {
    double h = 0.0;
    if (cudaMemcpyAsync(&h, nv.loss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return FT_ERR_CUDA;
    *loss_out = h / double(rows);
  }
  return FT_OK;
}

ft_status ft_stepnet_get(const void *net, int which, float *out_host, void *stream) {
  if (!net || !aligned16(net) || !out_host || which < 0 || which > 2) return FT_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const NetView nv = view(const_cast<void *>(net));
  if (which == 0 || which == 2) {
    const float *src = which == 0 ? nv.master : nv.last;
    if (cudaMemcpyAsync(out_host, src, sizeof(float) * NP, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return FT_ERR_CUDA;
    return FT_OK;
  }
  __nv_bfloat16 tmp[NP];
  if (cudaMemcpyAsync(tmp, nv.w, sizeof(__nv_bfloat16) * NP, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FT_ERR_CUDA;
  for (int q = 0; q < NP; ++q) out_host[q] = __bfloat162float(tmp[q]);
  return FT_OK;
}

}  // extern "C"
